// Streaming tall-skinny products over X - S (Algorithm 1, lines 5-6) and
// their split-K reduction, Gram partials and r x r right-multiplication.
//
// The product kernel streams the dense m x n matrix once per call; each CTA
// owns a 128-wide slab of the output dimension and one K-range, stages
// 128 x 32 tiles of Z (and the matching 32 x RP slice of the skinny
// operand) in shared memory with a register prefetch of the next tile, and
// accumulates an 8 x (RP/8) register tile per thread.
#include <cuda_bf16.h>

#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int TM = 128;   // output rows per CTA
constexpr int KC = 32;    // K per stage
constexpr int PASS_THREADS = 128;

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float4 ld4_bf16(const __nv_bfloat16* p) {
  uint2 u = *reinterpret_cast<const uint2*>(p);
  __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x);
  __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
  float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <typename T>
__device__ __forceinline__ float4 load_z4(const T* Z, int64_t row, int64_t col, int64_t m, int64_t n,
                                          int64_t ldz) {
  // 4 consecutive elements Z[row][col..col+3]; zero outside [0,m) x [0,n).
  if (row >= m || col >= n) return make_float4(0.f, 0.f, 0.f, 0.f);
  const T* p = Z + row * ldz + col;
  if (col + 4 <= n) {
    if constexpr (sizeof(T) == 4) return ld4(reinterpret_cast<const float*>(p));
    else return ld4_bf16(reinterpret_cast<const __nv_bfloat16*>(p));
  }
  float v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (col + c < n) {
      if constexpr (sizeof(T) == 4) v[c] = reinterpret_cast<const float*>(p)[c];
      else v[c] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[c]);
    } else {
      v[c] = 0.f;
    }
  }
  return make_float4(v[0], v[1], v[2], v[3]);
}

// TRANS = false: part = Z[rows o0..o0+127, K-range] * B[K-range, :]   (out = rows of Z)
// TRANS = true : part = Z[K-range, cols o0..o0+127]^T * B[K-range, :] (out = cols of Z)
template <int RN, bool TRANS, typename T>
__global__ void __launch_bounds__(PASS_THREADS)
k_pass(const T* __restrict__ Z, int64_t m, int64_t n, int64_t ldz, const float* __restrict__ B,
       float* __restrict__ part, int splits, int64_t kchunk, const Ctl* ctl) {
  constexpr int RP = RN * 8;
  if (ctl && ctl->abort) return;
  __shared__ __align__(16) float Zs[KC][TM + 4];
  __shared__ __align__(16) float Bs[KC][RP];

  const int tid = threadIdx.x;
  const int split = blockIdx.x % splits;
  const int64_t o0 = (int64_t)(blockIdx.x / splits) * TM;
  const int64_t outdim = TRANS ? n : m;
  const int64_t K = TRANS ? m : n;
  const int64_t k0 = (int64_t)split * kchunk;
  const int64_t k1 = min(K, k0 + kchunk);

  // Z tile loader mapping (8 float4 per thread per stage).
  float4 zr[8];
  float4 br[(KC * RP / 4 + PASS_THREADS - 1) / PASS_THREADS];
  constexpr int BR = (KC * RP / 4 + PASS_THREADS - 1) / PASS_THREADS;

  auto load_stage = [&](int64_t kb) {
    if (!TRANS) {
      // Tile rows o0..o0+127, cols kb..kb+31: two threads per 32-byte row piece.
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        int li = (s >> 2) * 64 + (tid >> 1);           // row within tile (0..127)
        int kk4 = (s & 3) * 2 + (tid & 1);             // float4 column (0..7)
        int64_t col = kb + kk4 * 4;
        zr[s] = (col < k1) ? load_z4(Z, o0 + li, col, m, min(n, k1), ldz) : make_float4(0, 0, 0, 0);
      }
    } else {
      // Tile rows kb..kb+31 (K), cols o0..o0+127: one warp per row, 32 float4.
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        int kk = s * 4 + (tid >> 5);
        int c4 = tid & 31;
        int64_t row = kb + kk;
        zr[s] = (row < k1) ? load_z4(Z, row, o0 + c4 * 4, m, n, ldz) : make_float4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int s = 0; s < BR; ++s) {
      int e = s * PASS_THREADS + tid;                  // float4 index in the KC x RP slice
      if (e < KC * RP / 4) {
        int kk = e / (RP / 4);
        int c4 = e % (RP / 4);
        int64_t krow = kb + kk;
        br[s] = (krow < k1) ? ld4(B + krow * RP + c4 * 4) : make_float4(0, 0, 0, 0);
      }
    }
  };
  auto store_stage = [&]() {
    if (!TRANS) {
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        int li = (s >> 2) * 64 + (tid >> 1);
        int kk4 = (s & 3) * 2 + (tid & 1);
        Zs[kk4 * 4 + 0][li] = zr[s].x;
        Zs[kk4 * 4 + 1][li] = zr[s].y;
        Zs[kk4 * 4 + 2][li] = zr[s].z;
        Zs[kk4 * 4 + 3][li] = zr[s].w;
      }
    } else {
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        int kk = s * 4 + (tid >> 5);
        int c4 = tid & 31;
        *reinterpret_cast<float4*>(&Zs[kk][c4 * 4]) = zr[s];
      }
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
    __syncthreads();                 // previous stage fully consumed
    store_stage();
    __syncthreads();
    if (kb + KC < k1) load_stage(kb + KC);   // next tile in flight during the FMAs
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

  float* out = part + (int64_t)split * outdim * RP;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int64_t o = o0 + ty * 8 + a;
    if (o < outdim) {
#pragma unroll
      for (int c = 0; c < RN; ++c) out[o * RP + tx + 8 * c] = acc[a][c];
    }
  }
}

template <bool TRANS, typename T>
void launch_pass_t(const PassArgs& a, cudaStream_t st) {
  const int64_t outdim = TRANS ? a.n : a.m;
  const int64_t tiles = (outdim + TM - 1) / TM;
  dim3 grid((unsigned)(tiles * a.splits));
  const T* Z = reinterpret_cast<const T*>(a.Z);
#define GODEC_PASS_CASE(RNV)                                                                  \
  case RNV:                                                                                   \
    k_pass<RNV, TRANS, T><<<grid, PASS_THREADS, 0, st>>>(Z, a.m, a.n, a.ldz, a.B, a.part,     \
                                                          a.splits, a.kchunk, a.ctl);         \
    break;
  switch (a.RP / 8) {
    GODEC_PASS_CASE(1)
    GODEC_PASS_CASE(2)
    GODEC_PASS_CASE(3)
    GODEC_PASS_CASE(4)
    GODEC_PASS_CASE(5)
    GODEC_PASS_CASE(6)
    GODEC_PASS_CASE(7)
    GODEC_PASS_CASE(8)
    default: break;
  }
#undef GODEC_PASS_CASE
}

// ----------------------------------------------------------------------------------
// Split-K reduction in a fixed order, plus Gram partials of 64-row blocks.
// ----------------------------------------------------------------------------------
constexpr int RB = 64;   // rows per reduce block

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__global__ void __launch_bounds__(256)
k_reduce(const float* __restrict__ part, int splits, int64_t rows, int RP, float* __restrict__ out,
         void* gram_part, int gram_mode, const Ctl* ctl) {
  if (ctl && ctl->abort) return;
  __shared__ float Ps[RB][kMaxRP + 1];
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  const int nrow = (int)(rows - r0 < RB ? rows - r0 : RB);
  const int tid = threadIdx.x;
  const int64_t stride = rows * RP;
  for (int e = tid; e < RB * RP; e += 256) {
    int i = e / RP, c = e % RP;
    float s = 0.f;
    if (i < nrow) {
      const float* p = part + (r0 + i) * RP + c;
      for (int sp = 0; sp < splits; ++sp) s += p[sp * stride];
      out[(r0 + i) * RP + c] = s;
    }
    Ps[i][c] = s;
  }
  if (gram_mode == 0) return;
  __syncthreads();
  const int npair = RP * RP;
  for (int e = tid; e < npair; e += 256) {
    int a = e / RP, c = e % RP;
    if (gram_mode == 1) {
      float g = 0.f;
      for (int i = 0; i < nrow; ++i) g = fmaf(Ps[i][a], Ps[i][c], g);
      reinterpret_cast<float*>(gram_part)[(int64_t)blockIdx.x * npair + e] = g;
    } else {
      // exact float32 products, double-float accumulation, stored as double
      float hi = 0.f, lo = 0.f;
      for (int i = 0; i < nrow; ++i) {
        float p, pe;
        two_prod(Ps[i][a], Ps[i][c], p, pe);
        float s = hi + p;
        float bb = s - hi;
        float err = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += err + pe;
      }
      reinterpret_cast<double*>(gram_part)[(int64_t)blockIdx.x * npair + e] = (double)hi + (double)lo;
    }
  }
}

// Q = P T with T (RP x RP) upper triangular or dense; optional float Gram partials.
__global__ void __launch_bounds__(256)
k_apply(const float* __restrict__ P, int64_t rows, int RP, const float* __restrict__ T, int upper,
        float* __restrict__ Q, float* __restrict__ gram_part, const Ctl* ctl) {
  if (ctl && ctl->abort) return;
  __shared__ float Ts[kMaxRP][kMaxRP + 1];
  __shared__ float Ps[RB][kMaxRP + 1];
  __shared__ float Qs[RB][kMaxRP + 1];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  const int nrow = (int)(rows - r0 < RB ? rows - r0 : RB);
  for (int e = tid; e < RP * RP; e += 256) Ts[e / RP][e % RP] = T[e];
  for (int e = tid; e < RB * RP; e += 256) {
    int i = e / RP, c = e % RP;
    Ps[i][c] = (i < nrow) ? P[(r0 + i) * RP + c] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < RB * RP; e += 256) {
    int i = e / RP, c = e % RP;
    float s = 0.f;
    const int amax = upper ? c : RP - 1;
    for (int a = 0; a <= amax; ++a) s = fmaf(Ps[i][a], Ts[a][c], s);
    Qs[i][c] = (i < nrow) ? s : 0.f;
    if (i < nrow) Q[(r0 + i) * RP + c] = s;
  }
  if (!gram_part) return;
  __syncthreads();
  for (int e = tid; e < RP * RP; e += 256) {
    int a = e / RP, c = e % RP;
    float g = 0.f;
    for (int i = 0; i < nrow; ++i) g = fmaf(Qs[i][a], Qs[i][c], g);
    gram_part[(int64_t)blockIdx.x * RP * RP + e] = g;
  }
}

}  // namespace

void pass_geometry(int64_t outdim, int64_t K, int nsm, int* splits, int64_t* kchunk) {
  const int64_t tiles = (outdim + TM - 1) / TM;
  // Aim at about 4 CTAs per SM, each with at least 256 values of K.
  int64_t want = (4LL * nsm + tiles - 1) / tiles;
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

void launch_pass(const PassArgs& a, cudaStream_t st) {
  if (a.bf16) {
    if (a.trans) launch_pass_t<true, __nv_bfloat16>(a, st);
    else launch_pass_t<false, __nv_bfloat16>(a, st);
  } else {
    if (a.trans) launch_pass_t<true, float>(a, st);
    else launch_pass_t<false, float>(a, st);
  }
}

int64_t reduce_blocks(int64_t rows) { return (rows + RB - 1) / RB; }

void launch_reduce(const float* part, int splits, int64_t rows, int RP, float* out, void* gram_part,
                   int gram_mode, const Ctl* ctl, cudaStream_t st) {
  k_reduce<<<(unsigned)reduce_blocks(rows), 256, 0, st>>>(part, splits, rows, RP, out, gram_part,
                                                           gram_mode, ctl);
}

void launch_apply(const float* P, int64_t rows, int RP, const float* T, int upper, float* Q,
                  float* gram_part, const Ctl* ctl, cudaStream_t st) {
  k_apply<<<(unsigned)reduce_blocks(rows), 256, 0, st>>>(P, rows, RP, T, upper, Q, gram_part, ctl);
}

}  // namespace godec
