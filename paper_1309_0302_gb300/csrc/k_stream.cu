// Streaming tall-skinny products over X - S (the power chain of Algorithm 1).
//
// Both products of the power chain, Z B and Z^T C, are computed as
// "row-major source times skinny matrix": Z^T C streams the transposed copy
// of X - S that the library keeps in HBM, so one kernel serves both.
//
// k_prod: each CTA owns a 128-row tile of the output and one K-range, stages
// 128 x 32 tiles of the source (and the matching 32 x RP slice of the skinny
// operand) in shared memory with a register prefetch of the next tile, and
// accumulates an 8 x (RP/8) register tile per thread.  The CTA that finishes a
// tile last (per-tile arrival counter) sums the split-K partials in split order
// (deterministic), optionally right-multiplies the rows by a normaliser T, writes
// the output rows and the tile's Gram partial Q^T Q for the next orthonormalisation.
#include <cuda_bf16.h>

#include <cuda_fp16.h>

#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int TM = 128;   // output rows per CTA
constexpr int KC = 32;    // K per stage
constexpr int PASS_THREADS = 128;
constexpr int EPI_STRIDE = kMaxRP + 1;
// stage buffers (KC x (TM+4) + KC x 64 floats) or the epilogue (TM + 64 rows of EPI_STRIDE)
constexpr size_t kProdSmem = (size_t)(TM + kMaxRP) * EPI_STRIDE * sizeof(float);

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float4 ld4_bf16(const __nv_bfloat16* p) {
  uint2 u = *reinterpret_cast<const uint2*>(p);
  __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x);
  __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
  float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <typename T>
__device__ __forceinline__ float4 load_z4(const T* Z, int64_t row, int64_t col, int64_t rows, int64_t kend,
                                          int64_t ld) {
  // 4 consecutive elements Z[row][col..col+3]; zero outside [0,rows) x [0,kend).
  if (row >= rows || col >= kend) return make_float4(0.f, 0.f, 0.f, 0.f);
  const T* p = Z + row * ld + col;
  if (col + 4 <= kend) {
    if constexpr (sizeof(T) == 4) return ld4(reinterpret_cast<const float*>(p));
    else return ld4_bf16(reinterpret_cast<const __nv_bfloat16*>(p));
  }
  float v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (col + c < kend) {
      if constexpr (sizeof(T) == 4) v[c] = reinterpret_cast<const float*>(p)[c];
      else v[c] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[c]);
    } else {
      v[c] = 0.f;
    }
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// Gram partial of the rows in Ps (nrow x RP, stride EPI_STRIDE): float, or exact
// float32 products summed in double-float and stored as double.
__device__ void tile_gram(const float* Ps, int nrow, int RP, int gram_mode, void* out, int nthreads) {
  const int npair = RP * RP;
  for (int e = threadIdx.x; e < npair; e += nthreads) {
    const int a = e / RP, c = e % RP;
    if (gram_mode == 1) {
      float g0 = 0.f, g1 = 0.f;
      int i = 0;
      for (; i + 1 < nrow; i += 2) {
        g0 = fmaf(Ps[i * EPI_STRIDE + a], Ps[i * EPI_STRIDE + c], g0);
        g1 = fmaf(Ps[(i + 1) * EPI_STRIDE + a], Ps[(i + 1) * EPI_STRIDE + c], g1);
      }
      if (i < nrow) g0 = fmaf(Ps[i * EPI_STRIDE + a], Ps[i * EPI_STRIDE + c], g0);
      reinterpret_cast<float*>(out)[e] = g0 + g1;
    } else {
      float hi = 0.f, lo = 0.f;
      for (int i = 0; i < nrow; ++i) {
        float p, pe;
        two_prod(Ps[i * EPI_STRIDE + a], Ps[i * EPI_STRIDE + c], p, pe);
        float s = hi + p;
        float bb = s - hi;
        float err = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += err + pe;
      }
      reinterpret_cast<double*>(out)[e] = (double)hi + (double)lo;
    }
  }
}

// part = Zsrc[rows o0..o0+127, K-range] * B[K-range, :], then the fused epilogue.
template <int RN, typename T>
__global__ void __launch_bounds__(PASS_THREADS)
k_prod(const T* __restrict__ Z, int64_t rows, int64_t K, int64_t ld, const float* __restrict__ B,
       float* __restrict__ part, int splits, int64_t kchunk, unsigned* __restrict__ counters,
       float* __restrict__ out, const float* __restrict__ Tn0, const float* __restrict__ Tn1, void* gram_part,
       int gram_mode, const Ctl* ctl) {
  constexpr int RP = RN * 8;
  if (ctl && ctl->abort) return;
  const float* Tn = (ctl && ctl->slot_parity) ? Tn1 : Tn0;
  extern __shared__ __align__(16) float sm[];
  float (*Zs)[TM + 4] = reinterpret_cast<float (*)[TM + 4]>(sm);       // [KC][TM+4]
  float (*Bs)[RP] = reinterpret_cast<float (*)[RP]>(sm + KC * (TM + 4)); // [KC][RP]

  const int tid = threadIdx.x;
  const int tile = blockIdx.x / splits;
  const int split = blockIdx.x % splits;
  const int64_t o0 = (int64_t)tile * TM;
  const int64_t k0 = (int64_t)split * kchunk;
  const int64_t k1 = min(K, k0 + kchunk);

  float4 zr[8];
  constexpr int BR = (KC * RP / 4 + PASS_THREADS - 1) / PASS_THREADS;
  float4 br[BR];

  auto load_stage = [&](int64_t kb) {
    // 128 rows x 32 columns: two threads per 32-byte row piece.
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int li = (s >> 2) * 64 + (tid >> 1);
      int kk4 = (s & 3) * 2 + (tid & 1);
      zr[s] = load_z4(Z, o0 + li, kb + kk4 * 4, rows, k1, ld);
    }
#pragma unroll
    for (int s = 0; s < BR; ++s) {
      int e = s * PASS_THREADS + tid;
      if (e < KC * RP / 4) {
        int kk = e / (RP / 4);
        int c4 = e % (RP / 4);
        int64_t krow = kb + kk;
        br[s] = (krow < k1) ? ld4(B + krow * RP + c4 * 4) : make_float4(0, 0, 0, 0);
      }
    }
  };
  auto store_stage = [&]() {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int li = (s >> 2) * 64 + (tid >> 1);
      int kk4 = (s & 3) * 2 + (tid & 1);
      Zs[kk4 * 4 + 0][li] = zr[s].x;
      Zs[kk4 * 4 + 1][li] = zr[s].y;
      Zs[kk4 * 4 + 2][li] = zr[s].z;
      Zs[kk4 * 4 + 3][li] = zr[s].w;
    }
#pragma unroll
    for (int s = 0; s < BR; ++s) {
      int e = s * PASS_THREADS + tid;
      if (e < KC * RP / 4) {
        int kk = e / (RP / 4);
        int c4 = e % (RP / 4);
        *reinterpret_cast<float4*>(&Bs[kk][c4 * 4]) = br[s];
      }
    }
  };

  const int ty = tid >> 3;   // 16 row groups of 8 output rows
  const int tx = tid & 7;    // 8 column groups, columns tx + 8c
  float acc[8][RN];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < RN; ++c) acc[a][c] = 0.f;

  if (k0 < k1) load_stage(k0);
  for (int64_t kb = k0; kb < k1; kb += KC) {
    __syncthreads();
    store_stage();
    __syncthreads();
    if (kb + KC < k1) load_stage(kb + KC);
#pragma unroll 8
    for (int kk = 0; kk < KC; ++kk) {
      float4 a0 = *reinterpret_cast<const float4*>(&Zs[kk][ty * 8]);
      float4 a1 = *reinterpret_cast<const float4*>(&Zs[kk][ty * 8 + 4]);
      float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[RN];
#pragma unroll
      for (int c = 0; c < RN; ++c) bv[c] = Bs[kk][tx + 8 * c];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < RN; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
    }
  }

  // ---- split-K partial, then the last CTA of the tile finishes it ----------------
  const int nrow = (int)(rows - o0 < TM ? rows - o0 : TM);
  float* mine = part + ((int64_t)split * rows + o0) * RP;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int i = ty * 8 + a;
    if (i < nrow) {
#pragma unroll
      for (int c = 0; c < RN; ++c) mine[(int64_t)i * RP + tx + 8 * c] = acc[a][c];
    }
  }
  __threadfence();
  __syncthreads();
  __shared__ unsigned s_last;
  if (tid == 0) s_last = (atomicAdd(&counters[tile], 1u) == (unsigned)splits - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) counters[tile] = 0u;          // ready for the next product
  float* Ps = sm;                              // [TM][EPI_STRIDE], reuses the stage buffers
  float* Ts = sm + TM * EPI_STRIDE;            // [RP][EPI_STRIDE]
  for (int e = tid; e < TM * RP; e += PASS_THREADS) {
    const int i = e / RP, c = e % RP;
    float s = 0.f;
    if (i < nrow) {
      const float* p = part + (o0 + i) * RP + c;
      for (int sp = 0; sp < splits; ++sp) s += __ldcg(p + (int64_t)sp * rows * RP);
    }
    Ps[i * EPI_STRIDE + c] = s;
  }
  if (Tn) {
    for (int e = tid; e < RP * RP; e += PASS_THREADS) Ts[(e / RP) * EPI_STRIDE + e % RP] = Tn[e];
    __syncthreads();
    // Q = P T: thread owns row `tid` (128 rows, 128 threads)
    float q[RP];
#pragma unroll
    for (int c = 0; c < RP; ++c) q[c] = 0.f;
    for (int a = 0; a < RP; ++a) {
      const float pa = Ps[tid * EPI_STRIDE + a];
#pragma unroll
      for (int c = 0; c < RP; ++c) q[c] = fmaf(pa, Ts[a * EPI_STRIDE + c], q[c]);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < RP; ++c) Ps[tid * EPI_STRIDE + c] = (tid < nrow) ? q[c] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < nrow * RP; e += PASS_THREADS)
    out[(o0 + e / RP) * RP + e % RP] = Ps[(e / RP) * EPI_STRIDE + e % RP];
  if (gram_mode) {
    const size_t stride = (size_t)RP * RP * (gram_mode == 2 ? 8 : 4);
    tile_gram(Ps, nrow, RP, gram_mode, reinterpret_cast<char*>(gram_part) + (size_t)tile * stride,
              PASS_THREADS);
  }
}

template <typename T>
void launch_prod_t(const ProdArgs& a, cudaStream_t st) {
  const int64_t tiles = (a.rows + TM - 1) / TM;
  dim3 grid((unsigned)(tiles * a.splits));
  const T* Z = reinterpret_cast<const T*>(a.Z);
#define GODEC_PROD_CASE(RNV)                                                                        \
  case RNV:                                                                                         \
    k_prod<RNV, T><<<grid, PASS_THREADS, kProdSmem, st>>>(Z, a.rows, a.K, a.ld, a.B, a.part,        \
                                                          a.splits, a.kchunk, a.counters, a.out,    \
                                                          a.Tn[0], a.Tn[1], a.gram_part,            \
                                                          a.gram_mode, a.ctl);                      \
    break;
  switch (a.RP / 8) {
    GODEC_PROD_CASE(1)
    GODEC_PROD_CASE(2)
    GODEC_PROD_CASE(3)
    GODEC_PROD_CASE(4)
    GODEC_PROD_CASE(5)
    GODEC_PROD_CASE(6)
    GODEC_PROD_CASE(7)
    GODEC_PROD_CASE(8)
    default: break;
  }
#undef GODEC_PROD_CASE
}

template <typename T>
cudaError_t prepare_prod_t() {
  cudaError_t e = cudaSuccess;
#define GODEC_PREP(RNV)                                                                                   \
  if (e == cudaSuccess)                                                                                   \
    e = cudaFuncSetAttribute(k_prod<RNV, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProdSmem);
  GODEC_PREP(1) GODEC_PREP(2) GODEC_PREP(3) GODEC_PREP(4) GODEC_PREP(5) GODEC_PREP(6) GODEC_PREP(7) GODEC_PREP(8)
#undef GODEC_PREP
  return e;
}

// ----------------------------------------------------------------------------------
// Q = P T (T dense RP x RP; a triangular inverse is passed as a dense matrix), for
// rows x RP row-major P.  64 rows per block; thread (g, c) keeps column c of T in registers
// and forms Q[i][c] for the rows i = g mod (256 / RPc) of the block (RPc = RP rounded up
// to 16, 32 or 64), reading each row of P as float4
// broadcasts (one shared-memory wavefront per four fmas of the warp; staging T per thread
// row instead re-reads it for every row and leaves the kernel bound by shared memory).
// The block's rows are staged in shared memory before any output is written, so P and Q
// may alias.  Optional outputs: Q itself, the float16 split transposed copy for the
// tensor-core product, and the block's float Gram partial QᵀQ.
// ----------------------------------------------------------------------------------
constexpr int RB = 64;              // rows per block
constexpr int AP_THREADS = 256;
constexpr int AP_OLD = kMaxRP + 1;  // T, then the output rows: odd stride, column reads conflict-free

// RPc: RP rounded up to 16, 32 or 64 (thread (g, c): column c < RPc of rows g + (256 / RPc) k).
template <int RPc>
__global__ void __launch_bounds__(AP_THREADS)
k_apply(const float* P, int64_t rows, int RP, const float* __restrict__ T0, const float* __restrict__ T1, float* Q,
        float* __restrict__ gram_part, const Ctl* ctl, void* __restrict__ bt2, int64_t ldb) {
  constexpr int PLD = RPc + 4;                 // P rows: float4-aligned (read as broadcasts)
  constexpr int NG = AP_THREADS / RPc;         // row groups
  constexpr int RPT = RB / NG;                 // rows per thread
  if (ctl && ctl->abort) return;
  const float* T = (ctl && ctl->slot_parity) ? T1 : T0;
  __shared__ float Ts[kMaxRP * AP_OLD];   // T, then the output rows
  __shared__ __align__(16) float Ps[RB * PLD];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  const int nrow = (int)(rows - r0 < RB ? rows - r0 : RB);
  // Every load is issued before the first store (T and the block's rows as float4s: RP is
  // a multiple of 8), so the block waits for one memory round trip, not one per element.
  constexpr int kT4 = (RPc * RPc / 4 + AP_THREADS - 1) / AP_THREADS, kP4 = RB * RPc / 4 / AP_THREADS;
  const int RP4 = RP / 4, nT4 = RP * RP4, nP4 = nrow * RP4;
  const float4* T4 = reinterpret_cast<const float4*>(T);
  const float4* P4 = reinterpret_cast<const float4*>(P + r0 * RP);
  float4 tv[kT4], pv[kP4];
#pragma unroll
  for (int k = 0; k < kT4; ++k) {
    const int e = tid + k * AP_THREADS;
    tv[k] = e < nT4 ? __ldg(T4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < kP4; ++k) {
    const int e = tid + k * AP_THREADS;
    pv[k] = e < nP4 ? __ldcg(P4 + e) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // T rows and P rows into shared memory; P's columns RP .. RPc-1 and rows past nrow zero
#pragma unroll
  for (int k = 0; k < kT4; ++k) {
    const int e = tid + k * AP_THREADS;
    if (e < nT4) {
      float* t = Ts + (e / RP4) * AP_OLD + (e % RP4) * 4;
      t[0] = tv[k].x;
      t[1] = tv[k].y;
      t[2] = tv[k].z;
      t[3] = tv[k].w;
    }
  }
#pragma unroll
  for (int k = 0; k < kP4; ++k) {
    const int e = tid + k * AP_THREADS;   // float4 e of the block's rows (row e / RP4)
    if (e < RB * RP4) *reinterpret_cast<float4*>(Ps + (e / RP4) * PLD + (e % RP4) * 4) = pv[k];
  }
  const int pad4 = RPc / 4 - RP4;
  for (int e = tid; e < RB * pad4; e += AP_THREADS)
    *reinterpret_cast<float4*>(Ps + (e / pad4) * PLD + (RP4 + e % pad4) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const int c = tid % RPc, g = tid / RPc;
  float tcol[RPc];
#pragma unroll
  for (int a = 0; a < RPc; ++a) tcol[a] = (a < RP && c < RP) ? Ts[a * AP_OLD + c] : 0.f;
  float acc[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) acc[k] = 0.f;
#pragma unroll
  for (int a = 0; a < RPc; a += 4) {
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
      const float4 p = *reinterpret_cast<const float4*>(Ps + (g + NG * k) * PLD + a);
      acc[k] = fmaf(p.x, tcol[a], acc[k]);
      acc[k] = fmaf(p.y, tcol[a + 1], acc[k]);
      acc[k] = fmaf(p.z, tcol[a + 2], acc[k]);
      acc[k] = fmaf(p.w, tcol[a + 3], acc[k]);
    }
  }
  __syncthreads();   // every thread has read T: Ts takes the output rows
  float* Os = Ts;
  if (c < RP)
#pragma unroll
    for (int k = 0; k < RPT; ++k) Os[(g + NG * k) * AP_OLD + c] = acc[k];
  __syncthreads();
  if (Q)
    for (int e = tid; e < nrow * RP; e += AP_THREADS) {
      const int i = e / RP, cc = e % RP;
      Q[(r0 + i) * RP + cc] = Os[i * AP_OLD + cc];
    }
  if (bt2) {
    __half* b2 = reinterpret_cast<__half*>(bt2);
    for (int e = tid; e < RP * RB; e += AP_THREADS) {
      const int cc = e / RB, i = e % RB;   // consecutive threads: consecutive rows of one column
      if (i < nrow) {
        const float v = Os[i * AP_OLD + cc] * kSkinnyScale;
        const __half c1 = __float2half_rn(v);
        b2[(int64_t)cc * ldb + r0 + i] = c1;
        b2[(int64_t)(RP + cc) * ldb + r0 + i] = __float2half_rn((v - __half2float(c1)) * 2048.f);
      }
    }
  }
  if (!gram_part) return;
  // Gram partial: thread (bi, bj) accumulates the 4 x 4 block rows 4bi.., columns 4bj..
  const int bi = tid >> 4, bj = tid & 15;
  float gg[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) gg[u][v] = 0.f;
  if (4 * bi < RP && 4 * bj < RP) {
#pragma unroll 4
    for (int i = 0; i < nrow; ++i) {
      float x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        x[u] = Os[i * AP_OLD + 4 * bi + u];
        y[u] = Os[i * AP_OLD + 4 * bj + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) gg[u][v] = fmaf(x[u], y[v], gg[u][v]);
    }
    float* out = gram_part + (int64_t)blockIdx.x * RP * RP;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) out[(4 * bi + u) * RP + 4 * bj + v] = gg[u][v];
  }
}

}  // namespace

void prod_geometry(int64_t rows, int64_t K, int nsm, int* splits, int64_t* kchunk) {
  const int64_t tiles = (rows + TM - 1) / TM;
  // Aim at about 3 CTAs per SM, each with at least 256 values of K.
  int64_t want = (3LL * nsm + tiles - 1) / tiles;
  int64_t maxs = (K + 255) / 256;
  int64_t s = want < 1 ? 1 : want;
  if (s > maxs) s = maxs < 1 ? 1 : maxs;
  int64_t ch = (K + s - 1) / s;
  ch = ((ch + KC - 1) / KC) * KC;
  s = (K + ch - 1) / ch;
  if (s < 1) s = 1;
  *splits = (int)s;
  *kchunk = ch;
}

int64_t prod_tiles(int64_t rows) { return (rows + TM - 1) / TM; }

void launch_prod(const ProdArgs& a, cudaStream_t st) {
  if (a.bf16) launch_prod_t<__nv_bfloat16>(a, st);
  else launch_prod_t<float>(a, st);
}

cudaError_t prepare_stream_kernels() {
  cudaError_t e = prepare_prod_t<float>();
  if (e == cudaSuccess) e = prepare_prod_t<__nv_bfloat16>();
  return e;
}

int64_t apply_blocks(int64_t rows) { return (rows + RB - 1) / RB; }

void launch_apply(const float* P, int64_t rows, int RP, const float* T0, const float* T1, float* Q,
                  float* gram_part, const Ctl* ctl, cudaStream_t st, void* bt2, int64_t ldb) {
  const unsigned grid = (unsigned)apply_blocks(rows);
  if (RP <= 16) k_apply<16><<<grid, AP_THREADS, 0, st>>>(P, rows, RP, T0, T1, Q, gram_part, ctl, bt2, ldb);
  else if (RP <= 32) k_apply<32><<<grid, AP_THREADS, 0, st>>>(P, rows, RP, T0, T1, Q, gram_part, ctl, bt2, ldb);
  else k_apply<64><<<grid, AP_THREADS, 0, st>>>(P, rows, RP, T0, T1, Q, gram_part, ctl, bt2, ldb);
}

}  // namespace godec
