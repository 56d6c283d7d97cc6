// r x r kernels of the L-step (one thread block each, except the Gram sums).
//
// Eq. (mlr_app) needs the QR factors of the power chain and an r x r core
// M = R1 (A2^T Y1)^{-1} R2^T with an SVD for its (2q+1)-th root.  With
// Q2 = orth(Y2), L~ Q2 = Q1 R_{2q} ... R_0, and since A2^T Y1 = R2^T R2 the
// core equals that product of R factors (up to the row basis of Q1).  The
// chain is orthonormalised by Cholesky factors of Gram matrices (CholeskyQR);
// every product of chain 3 contributes the factor it was normalised with.
//
// GB300's float64 rate is a small fraction of its float32 rate: a float64 Cholesky of a
// 56 x 56 Gram takes about 110 us on one SM against 31 us for the blocked float32 one.
// float64 is used for the Gram sums over row tiles and the rank test (a pivoted Cholesky
// on an exactly accumulated Gram).  The Cholesky factors of the critical-path
// orthonormalisations (k_chol) run in float32 by default and in float64 with
// GODEC_FLAG_FP64_FACTOR; the factor is applied in float32 either way.  The lagged
// normalisers (k_slot, off the critical path) and the core SVD run in float32.
#include <math.h>

#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int SMALL_THREADS = 256;   // 16 x 16 threads, each owning a 4 x 4 block of 64 x 64
constexpr int LD = kMaxRP + 1;

// ---- Gram sums over row tiles --------------------------------------------------------
// Block = E entries x (NT / E) tile strides: each thread sums every (NT / E)-th partial of
// one entry in four independent chains, and the block adds the strides' sums by a fixed
// tree, so the order is fixed for given (nblk, E, NT).  Few entries (small r) take a
// small E and large blocks, so that many threads share the partials of each entry.
template <typename T, int E, int NT>
__global__ void __launch_bounds__(NT)
k_gram_sum(const T* __restrict__ part, int64_t nblk, int npair, double* __restrict__ out, float* __restrict__ out32,
           const Ctl* ctl) {
  if (ctl && ctl->abort) return;
  constexpr int SPLIT = NT / E;
  __shared__ double red[SPLIT][E];
  const int lane = threadIdx.x % E, sp = threadIdx.x / E;
  const int e = blockIdx.x * E + lane;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  if (e < npair) {
    int64_t b = sp;
    for (; b + 3 * SPLIT < nblk; b += 4 * SPLIT) {
      s0 += (double)part[b * npair + e];
      s1 += (double)part[(b + SPLIT) * npair + e];
      s2 += (double)part[(b + 2 * SPLIT) * npair + e];
      s3 += (double)part[(b + 3 * SPLIT) * npair + e];
    }
    for (; b < nblk; b += SPLIT) s0 += (double)part[b * npair + e];
  }
  red[sp][lane] = (s0 + s1) + (s2 + s3);
  __syncthreads();
#pragma unroll
  for (int h = SPLIT / 2; h >= 1; h >>= 1) {
    if (sp < h) red[sp][lane] += red[sp + h][lane];
    __syncthreads();
  }
  if (sp == 0 && e < npair) {
    const double t = red[0][lane];
    out[e] = t;
    if (out32) out32[e] = (float)t;   // the float copy: its reader then needs no float64 work
  }
}

// ---- block helpers on 64 x 64 (padded RP x RP) matrices in shared memory -----------
// Thread (ty, tx) owns rows ty + 16a and columns tx + 16b, a, b in 0..3.

constexpr int CB = 8;   // block size of the triangular inverse

// Inverse of the 8 x 8 upper-triangular block at (k0, k0) of R into Ui (lane c < 8
// back-substitutes column c; rd[i] = 1 / R[k0+i][k0+i]).
__device__ __forceinline__ void block_inverse8(const float (*R)[LD], int k0, const float* rd, float (*Ui)[LD],
                                               int ui0, int lane) {
  if (lane < 8) {
    float x[8];
#pragma unroll
    for (int i = 7; i >= 0; --i) {
      float sacc = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int j = i + 1; j < 8; ++j) sacc = fmaf(-R[k0 + i][k0 + j], x[j], sacc);
      x[i] = (i <= lane) ? sacc * rd[i] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) Ui[ui0 + i][ui0 + lane] = x[i];
  }
}

// Inverse Ri of an upper-triangular R (n a multiple of 8), in 8 x 8 blocks: warps
// invert the diagonal blocks in parallel, then block diagonals d = 1, 2, ... follow from
// T_ij = -T_ii sum_{k=i+1..j} R_ik T_kj.  One thread per output entry: the 8 threads of
// a column (adjacent lanes) each form one entry of S = sum R_ik T_kj and exchange them
// by shuffles for the product with T_ii.  R must be visible to all threads on entry;
// Ri must not alias R.
__device__ void tri_inverse(const float (*R)[LD], float (*Ri)[LD], int n, float*) {
  __shared__ float rdg[kMaxRP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nb = n / CB;
  for (int e = tid; e < kMaxRP * kMaxRP; e += SMALL_THREADS) Ri[e / kMaxRP][e % kMaxRP] = 0.f;
  if (tid < n) rdg[tid] = 1.f / R[tid][tid];
  __syncthreads();
  for (int b = warp; b < nb; b += SMALL_THREADS / 32) block_inverse8(R, b * CB, rdg + b * CB, Ri, b * CB, lane);
  __syncthreads();
  for (int d = 1; d < nb; ++d) {
    const int nitem = (nb - d) * CB * CB;   // (block i, column of block i + d, row a)
    for (int base = tid - lane; base < nitem; base += SMALL_THREADS) {
      const int it = base + lane;
      const bool act = it < nitem;
      const int a = it & 7, cc = (it >> 3) & 7, bi = it >> 6;
      const int i0 = bi * CB, col = (bi + d) * CB + cc;
      float s0 = 0.f, s1 = 0.f;
      if (act) {
        int k = i0 + CB;
        for (; k + 1 <= col; k += 2) {
          s0 = fmaf(R[i0 + a][k], Ri[k][col], s0);
          s1 = fmaf(R[i0 + a][k + 1], Ri[k + 1][col], s1);
        }
        if (k <= col) s0 = fmaf(R[i0 + a][k], Ri[k][col], s0);
      }
      const float sv = s0 + s1;
      float tacc = 0.f;
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const float su = __shfl_sync(0xffffffffu, sv, u, 8);
        if (act) tacc = fmaf(Ri[i0 + a][i0 + u], su, tacc);
      }
      if (act) Ri[i0 + a][col] = -tacc;
    }
    __syncthreads();
  }
}

// C = A B (n x n, A upper triangular if a_upper); C may alias A or B.
__device__ void mat_mul(const float (*A)[LD], const float (*B)[LD], float (*C)[LD], int n, bool a_upper) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float acc[4][4];
#pragma unroll
  for (int ia = 0; ia < 4; ++ia)
#pragma unroll
    for (int ib = 0; ib < 4; ++ib) acc[ia][ib] = 0.f;
  for (int t = 0; t < n; ++t) {
    float av[4], bv[4];
#pragma unroll
    for (int ia = 0; ia < 4; ++ia) {
      const int a = ty + 16 * ia;
      av[ia] = (a < n && (!a_upper || t >= a)) ? A[a][t] : 0.f;
    }
#pragma unroll
    for (int ib = 0; ib < 4; ++ib) bv[ib] = B[t][tx + 16 * ib];
#pragma unroll
    for (int ia = 0; ia < 4; ++ia)
#pragma unroll
      for (int ib = 0; ib < 4; ++ib) acc[ia][ib] = fmaf(av[ia], bv[ib], acc[ia][ib]);
  }
  __syncthreads();
#pragma unroll
  for (int ia = 0; ia < 4; ++ia)
#pragma unroll
    for (int ib = 0; ib < 4; ++ib) C[ty + 16 * ia][tx + 16 * ib] = acc[ia][ib];
  __syncthreads();
}

// D = src (RP x RP, zero-padded to 64 x 64; src == nullptr gives the identity), with no
// closing barrier: several loads in flight, then one barrier.
// (256 threads: all sixteen loads of a thread are issued before the first store)
constexpr int kPerThread = kMaxRP * kMaxRP / SMALL_THREADS;
__device__ void load_mat_nb(float (*D)[LD], const float* src, int RP) {
  float v[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int e = threadIdx.x + k * SMALL_THREADS, i = e / kMaxRP, j = e % kMaxRP;
    if (src) v[k] = (i < RP && j < RP) ? __ldcg(src + i * RP + j) : 0.f;
    else v[k] = (i == j) ? 1.f : 0.f;
  }
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int e = threadIdx.x + k * SMALL_THREADS;
    D[e / kMaxRP][e % kMaxRP] = v[k];
  }
}

// Gram (double, RP x RP) into float G, padded block set to the identity, no closing
// barrier; *nf is set if the Gram holds NaN/Inf.
__device__ void load_gram_nb(float (*G)[LD], const double* g64, int r, int RP, int* nf) {
  double v[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int e = threadIdx.x + k * SMALL_THREADS, i = e / kMaxRP, j = e % kMaxRP;
    v[k] = (i < r && j < r) ? __ldcg(g64 + i * RP + j) : (i == j ? 1.0 : 0.0);
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int e = threadIdx.x + k * SMALL_THREADS;
    bad |= !isfinite(v[k]);
    G[e / kMaxRP][e % kMaxRP] = (float)v[k];
  }
  if (bad) *nf = 1;
}

// The same from the float copy of the Gram (written beside the float64 one by k_gram_sum):
// no float64 instruction, whose rate on GB300 would make these 4096 conversions and checks
// take microseconds on the one SM.
__device__ void load_gram32_nb(float (*G)[LD], const float* g32, int r, int RP, int* nf) {
  float v[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int e = threadIdx.x + k * SMALL_THREADS, i = e / kMaxRP, j = e % kMaxRP;
    v[k] = (i < r && j < r) ? __ldcg(g32 + i * RP + j) : (i == j ? 1.f : 0.f);
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int e = threadIdx.x + k * SMALL_THREADS;
    bad |= !isfinite(v[k]);
    G[e / kMaxRP][e % kMaxRP] = v[k];
  }
  if (bad) *nf = 1;
}

__device__ void store_mat(float* dst, const float (*S)[LD], int RP) {
  for (int e = threadIdx.x; e < RP * RP; e += SMALL_THREADS) dst[e] = S[e / RP][e % RP];
}

// Largest |M[i][j]| over the n x n block (all threads get it).
__device__ float block_absmax(const float (*M)[LD], int n) {
  __shared__ float red[32];   // one slot per warp of a block of up to 1024 threads
  float m = 0.f;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) m = fmaxf(m, fabsf(M[e / n][e % n]));
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
  __syncthreads();
  return r;
}

// Upper Cholesky factor and its inverse together, by symmetric Gaussian elimination of the
// augmented matrix [G | I] with one barrier per column.  With G = L D L^T (L unit lower),
// the elimination leaves U = D L^T in the left block and E = L^{-1} in the right one, so
// R = D^{-1/2} U and R^{-1} = E^T D^{-1/2}.  The trailing block is updated in full (both
// triangles), so column j holds the multipliers of step j.
// Thread (rw, cc) = (tid / 64, tid % 64) holds one column index cc and the rows of class rw
// (a = rw mod 4) not yet final, row rw + 4 (k + m) in register slot k (m rows of the class
// are final already): column cc of the left block until step cc, where the left column is
// done (its entries below the pivot are the multipliers, used in that step only) and the
// same registers take column cc of E over (I's column, zero in the rows kept).  Step j:
// the owners of row j (slot 0 of class j mod 4, final since step j-1) publish it as the
// pivot row, store it to Us / Es and shift it out of their registers (so every register
// index stays static); the pivot's owner publishes 1 / pivot; the owners of column j
// publish the multipliers' numerators, zero for the rows not updated.  After the barrier a
// step is one fma per register.  Only those rows and columns pass through shared memory
// (double-buffered, so one barrier a step), and no lane branches on its entries.  On return
// Us / Es (64 x LD) hold U and E by rows (columns < n).
constexpr int kRowsPT = kMaxRP / 4;

__device__ __forceinline__ void chol_reg_core(float (&V)[kRowsPT], int n, int nchk, float thr, int* bad, float* dv,
                                              float (*Us)[LD], float (*Es)[LD]) {
  __shared__ __align__(16) float prow[2][kMaxRP];   // row j: left entries (cc > j), E entries (cc <= j)
  __shared__ __align__(16) float pcol[2][kMaxRP];   // column j, slot k of class rw at rw * 16 + k
  __shared__ float pinv[2];
  const int tid = threadIdx.x, cc = tid & 63, rw = tid >> 6;
  for (int j = 0; j < n; ++j) {
    const int b = j & 1;
    const bool owner = rw == (j & 3);
    const int m = (j + 3 - rw) >> 2;   // rows of this class before row j, already shifted out
    if (owner && cc < n) {
      const float v0 = V[0];
      prow[b][cc] = (cc == j) ? 1.f : v0;
      Us[j][cc] = (cc >= j) ? v0 : 0.f;
      Es[j][cc] = (cc < j) ? v0 : ((cc == j) ? 1.f : 0.f);
      if (cc == j) {
        float d = v0;
        if (j < nchk && !(d > thr)) {
          d = thr > 0.f ? thr : 1e-30f;
          *bad = 1;
        }
        dv[j] = d;
        pinv[b] = 1.f / d;
      }
    }
    if (cc == j) {
#pragma unroll
      for (int k = 0; k < kRowsPT; k += 4) {
        float w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = rw + 4 * (k + u + m);
          w[u] = (a > j && a < n) ? V[k + u] : 0.f;
        }
        *reinterpret_cast<float4*>(&pcol[b][rw * 16 + k]) = make_float4(w[0], w[1], w[2], w[3]);
      }
#pragma unroll
      for (int k = 0; k < kRowsPT; ++k) V[k] = 0.f;   // column j of E from here on
    }
    __syncthreads();
    if (cc < n) {
      const float pj = prow[b][cc] * pinv[b];
#pragma unroll
      for (int k = 0; k < kRowsPT; k += 4) {
        const float4 m4 = *reinterpret_cast<const float4*>(&pcol[b][rw * 16 + k]);
        V[k] = fmaf(-m4.x, pj, V[k]);
        V[k + 1] = fmaf(-m4.y, pj, V[k + 1]);
        V[k + 2] = fmaf(-m4.z, pj, V[k + 2]);
        V[k + 3] = fmaf(-m4.w, pj, V[k + 3]);
      }
    }
    if (owner) {   // row j is out: the next row of this class moves to slot 0
#pragma unroll
      for (int k = 0; k + 1 < kRowsPT; ++k) V[k] = V[k + 1];
      V[kRowsPT - 1] = 0.f;
    }
  }
  __syncthreads();
}

// The same elimination of [G | I] by one warp, the matrix in registers: lane l holds
// columns l and l + 32 (all rows, RPc of them), G's column until its step, then E's (the
// registers of column j become E's column j at step j).  Step j: the pivot d = G[j][j] and
// the multipliers l_i = G[j][i] / d (row j of the columns i > j; G stays symmetric) are
// broadcast by shuffles, row j of U and E is stored, and every column takes
// x_i -= l_i x_j for i > j, column j itself becoming -l_i.  No block barrier: the steps
// are unrolled (RPc = RP rounded up to 16, 32 or 64; the padded block of G is the
// identity), so every register index is static.  Pivots j < nchk at or below thr are
// raised to thr and reported through *bad.
// Step j of chol_warp_core; the steps are instantiated one by one, so that every register
// index is a compile-time constant.
template <int RPc, int NS, int j>
__device__ __forceinline__ void chol_warp_step(float (&V)[NS][RPc], int lane, int nchk, float thr, int& badl, float* dv,
                                               float (*Us)[LD], float (*Es)[LD]) {
  if constexpr (j < RPc) {
    const unsigned full = 0xffffffffu;
    float d = __shfl_sync(full, V[j >> 5][j], j & 31);
    if (j < nchk && !(d > thr)) {
      d = thr > 0.f ? thr : 1e-30f;
      badl = 1;
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int c = lane + 32 * s;
      if (c < RPc) {
        const float v = V[s][j];
        Us[j][c] = c >= j ? v : 0.f;
        Es[j][c] = c < j ? v : (c == j ? 1.f : 0.f);
      }
    }
    if (lane == 0) dv[j] = d;
    const float inv = 1.f / d;
    const bool own = lane == (j & 31);   // this lane holds column j (in slot j >> 5)
#pragma unroll
    for (int i = j + 1; i < RPc; ++i) {
      const float li = __shfl_sync(full, V[i >> 5][j], i & 31) * inv;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const float upd = fmaf(-li, V[s][j], V[s][i]);
        V[s][i] = (s == (j >> 5) && own) ? -li : upd;
      }
    }
    chol_warp_step<RPc, NS, j + 1>(V, lane, nchk, thr, badl, dv, Us, Es);
  }
}

// The same elimination of [G | I] by one warp, the matrix in registers: lane l holds
// columns l and l + 32 (all rows, RPc of them), G's column until its step, then E's (the
// registers of column j become E's column j at step j).  Step j: the pivot d = G[j][j] and
// the multipliers l_i = G[j][i] / d (row j of the columns i > j; G stays symmetric) are
// broadcast by shuffles, row j of U and E is stored, and every column takes
// x_i -= l_i x_j for i > j, column j itself becoming -l_i.  No block barrier
// (RPc = RP rounded up to 16, 32 or 64; the padded block of G is the identity).  Pivots
// j < nchk at or below thr are raised to thr and reported through *bad.
template <int RPc>
__device__ __forceinline__ void chol_warp_core(const float (*G)[LD], float shift, int nchk, float thr, int* bad,
                                               float* dv, float (*Us)[LD], float (*Es)[LD]) {
  constexpr int NS = RPc > 32 ? 2 : 1;
  const int lane = threadIdx.x & 31;
  float V[NS][RPc];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int c = lane + 32 * s;
#pragma unroll
    for (int i = 0; i < RPc; ++i) V[s][i] = c < RPc ? G[i][c] + ((i == c && i < nchk) ? shift : 0.f) : 0.f;
  }
  int badl = 0;
  chol_warp_step<RPc, NS, 0>(V, lane, nchk, thr, badl, dv, Us, Es);
  if (lane == 0 && badl) *bad = 1;
}

// Cholesky with a shifted fallback: pivots below 1e-6 of the largest diagonal mean a
// numerically rank-deficient chain (Z of rank < r before the rank test lowers r); the
// factorisation is then redone on G + 1e-5 max(diag) I, which keeps Q bounded.  G (64 x 64,
// padded block the identity) is kept; on return Us / Es hold U and E (chol_reg_core) and
// dv the pivots used: R[a][c] = Us[a][c] / sqrt(dv[a]) (c > a), R[a][a] = sqrt(dv[a]),
// R^{-1}[i][c] = Es[c][i] / sqrt(dv[c]) (c >= i).
// WARP: RP <= 32, the one-warp elimination (instantiated apart, so that the kernels for
// larger RP do not carry its code).
template <bool WARP>
__device__ __forceinline__ void robust_chol(const float (*G)[LD], float (*Us)[LD], float (*Es)[LD], float* dv, int r,
                                            int RP, Ctl* ctl) {
  __shared__ float s_gmax;
  __shared__ int s_bad;
  const int tid = threadIdx.x, cc = tid & 63, rw = tid >> 6;
  if (tid < 32) {
    float gm = 0.f;
    for (int j = tid; j < r; j += 32) gm = fmaxf(gm, G[j][j]);
    for (int o = 16; o; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if (tid == 0) s_gmax = gm;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const float shift = attempt == 1 ? 1e-5f * s_gmax : 0.f;
    const float thr = 1e-6f * s_gmax;
    if constexpr (WARP) {
      // one warp, the matrix in registers (a fully unrolled elimination; above 32 columns
      // its straight-line code outgrows the instruction cache and the block version wins)
      if (tid < 32) {
        if (RP <= 16) chol_warp_core<16>(G, shift, r, thr, &s_bad, dv, Us, Es);
        else chol_warp_core<32>(G, shift, r, thr, &s_bad, dv, Us, Es);
      }
      __syncthreads();
    } else {
      float V[kRowsPT];
#pragma unroll
      for (int k = 0; k < kRowsPT; ++k) {
        const int a = rw + 4 * k;
        V[k] = G[a][cc] + ((a == cc && a < r) ? shift : 0.f);
      }
      chol_reg_core(V, RP, r, thr, &s_bad, dv, Us, Es);
    }
    if (!s_bad) break;
    if (tid == 0) ctl->chol_shifts += 1;
  }
}

// dst = M / max|M|, ctl->m_logscale (+)= log(max|M|).
__device__ void normalise_into(float (*M)[LD], float* dst, int RP, Ctl* ctl, bool reset_scale) {
  const float mx = block_absmax(M, RP);
  const float scale = mx > 0.f ? mx : 1.f;
  if (threadIdx.x == 0) ctl->m_logscale = (reset_scale ? 0.0 : ctl->m_logscale) + log((double)scale);
  const float inv = 1.f / scale;
  for (int e = threadIdx.x; e < RP * RP; e += SMALL_THREADS) dst[e] = M[e / RP][e % RP] * inv;
}

// float64 upper Cholesky G = R^T R of the RP x RP Gram in Gd (padded block = identity),
// right-looking, one column per barrier: the trailing update uses the unscaled pivot row
// (G[a][c] -= G[j][a] G[j][c] / G[j][j]), and the rows are scaled by 1 / sqrt(pivot) at
// the end.  Pivots j < r below thr are raised to thr and reported through *bad.  The
// float32 factor goes to R (lower triangle zero).
// GB300 issues a warp's float64 FMA over many cycles, so the trailing update runs over a
// dense list of the upper-triangle entries (a, c), a >= c's row, ordered by decreasing row
// a: the entries with a > j are the first (RP-1-j)(RP-j)/2 of the list, and no lane of a
// warp idles on a masked-out entry.  The list (tri, built by the caller) holds a << 8 | c.
__device__ void chol64(double (*Gd)[LD], float (*R)[LD], int r, int RP, double thr, int* bad,
                       const unsigned short* tri) {
  __shared__ double piv[kMaxRP];
  __shared__ double sc[kMaxRP];
  const int tid = threadIdx.x;
  for (int j = 0; j < RP; ++j) {
    const int w = RP - j - 1;
    // pivot and the scaled pivot row: sc[a] = G[j][a] / G[j][j]
    if (tid < kMaxRP) {
      double d = Gd[j][j];
      if (j < r && !(d > thr)) {
        if (tid == 0) *bad = 1;
        d = thr > 0.0 ? thr : 1e-300;
      }
      if (tid == 0) piv[j] = d;
      const int a = j + 1 + tid;
      if (tid < w) sc[a] = Gd[j][a] / d;
    }
    __syncthreads();
    const int nt = w * (w + 1) / 2;
    for (int e = tid; e < nt; e += SMALL_THREADS) {
      const int a = tri[e] >> 8, c = tri[e] & 255;
      Gd[a][c] = fma(-sc[a], Gd[j][c], Gd[a][c]);
    }
    __syncthreads();
  }
  for (int e = tid; e < kMaxRP * kMaxRP; e += SMALL_THREADS) {
    const int i = e / kMaxRP, c = e % kMaxRP;
    R[i][c] = (i < RP && c >= i && c < RP) ? (float)(Gd[i][c] / sqrt(piv[i])) : 0.f;
  }
  __syncthreads();
}

// ---- critical path: R from a Gram --------------------------------------------------------
// R (upper) with Rᵀ R = G and its inverse T = R^{-1}.  With alarm_ratio > 0 the
// factor of an almost orthonormal input is checked: a diagonal spread above the ratio
// means one CholeskyQR pass would not restore orthonormality, and the iteration is
// sent back to the exact path (alarm).
// F64: the factorisation runs in float64 (chol64) instead of the blocked float32 Cholesky;
// either way R and T = R^{-1} are stored in float32 and T is formed in float32.
template <bool F64, bool WARP>
__global__ void __launch_bounds__(SMALL_THREADS) k_chol(const double* __restrict__ g64, const float* __restrict__ g32,
                                                        int r, int RP,
                                                        float* __restrict__ Rout, float* __restrict__ Tout,
                                                        float alarm_ratio, Ctl* ctl) {
  if (ctl->abort) return;
  extern __shared__ __align__(16) float smf[];
  float (*R)[LD] = reinterpret_cast<float (*)[LD]>(smf) + 2 * kMaxRP;
  float (*Ri)[LD] = R + kMaxRP;
  __shared__ float dv[kMaxRP];
  if (!F64) {
    float (*G)[LD] = reinterpret_cast<float (*)[LD]>(smf);
    float (*E)[LD] = G + kMaxRP;
    int nf = 0;
    if (g32) load_gram32_nb(G, g32, r, RP, &nf);
    else load_gram_nb(G, g64, r, RP, &nf);
    if (__syncthreads_or(nf)) {
      if (threadIdx.x == 0) { ctl->nonfinite = 1; ctl->abort = 1; }
      return;
    }
    (void)E;
    robust_chol<WARP>(G, R, Ri, dv, r, RP, ctl);   // U into R's block, E into Ri's
  } else {
  double (*Gd)[LD] = reinterpret_cast<double (*)[LD]>(smf);            // 2 float blocks
  __shared__ double s_gmax;
  __shared__ int s_bad;
  __shared__ unsigned short tri[kMaxRP * (kMaxRP + 1) / 2];
  // upper-triangle entries (a, c), c >= a, of rows RP-1 down to 0 (see chol64)
  for (int e = threadIdx.x; e < RP * (RP + 1) / 2; e += SMALL_THREADS) {
    // e -> (a, c): rows from the bottom, row a = RP-1-k holding k+1 entries
    int k = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while (k * (k + 1) / 2 > e) --k;
    while ((k + 1) * (k + 2) / 2 <= e) ++k;
    const int a = RP - 1 - k, c = a + (e - k * (k + 1) / 2);
    tri[e] = (unsigned short)(a << 8 | c);
  }
  // the Gram in float64, padded block set to the identity; a non-finite Gram aborts
  int nf = 0;
  for (int e = threadIdx.x; e < kMaxRP * kMaxRP; e += SMALL_THREADS) {
    const int i = e / kMaxRP, j = e % kMaxRP;
    const double v = (i < r && j < r) ? __ldcg(g64 + i * RP + j) : (i == j ? 1.0 : 0.0);
    nf |= !isfinite(v);
  }
  if (__syncthreads_or(nf)) {
    if (threadIdx.x == 0) { ctl->nonfinite = 1; ctl->abort = 1; }
    return;
  }
  if (threadIdx.x == 0) {
    double gm = 0.0;
    for (int j = 0; j < r; ++j) gm = fmax(gm, __ldcg(g64 + j * RP + j));
    s_gmax = gm;
  }
  // Cholesky with a shifted fallback, as robust_chol
  for (int attempt = 0; attempt < 2; ++attempt) {
    __syncthreads();
    for (int e = threadIdx.x; e < kMaxRP * kMaxRP; e += SMALL_THREADS) {
      const int i = e / kMaxRP, j = e % kMaxRP;
      double v = (i < r && j < r) ? __ldcg(g64 + i * RP + j) : (i == j ? 1.0 : 0.0);
      if (attempt == 1 && i == j && i < r) v += 1e-5 * s_gmax;
      Gd[i][j] = v;
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    chol64(Gd, R, r, RP, 1e-6 * s_gmax, &s_bad, tri);
    if (!s_bad) break;
    if (threadIdx.x == 0) ctl->chol_shifts += 1;
  }
  __syncthreads();
  }
  if (alarm_ratio > 0.f && threadIdx.x < 32) {
    float lo = 3.4e38f, hi = 0.f;
    for (int j = threadIdx.x; j < r; j += 32) {
      const float dj = F64 ? R[j][j] : sqrtf(dv[j]);
      lo = fminf(lo, dj);
      hi = fmaxf(hi, dj);
    }
    for (int o = 16; o; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (threadIdx.x == 0 && !(hi <= alarm_ratio * lo)) { ctl->alarm = 1; ctl->abort = 1; }
  }
  if (!F64) {
    // R = D^{-1/2} U and T = E^T D^{-1/2} (U in R's block, E in Ri's)
    for (int e = threadIdx.x; e < RP * RP; e += SMALL_THREADS) {
      const int i = e / RP, c = e % RP;
      const float si = rsqrtf(dv[i]);
      Rout[e] = (c > i) ? R[i][c] * si : ((c == i) ? dv[i] * si : 0.f);
      Tout[e] = (c >= i) ? Ri[c][i] * rsqrtf(dv[c]) : 0.f;
    }
  } else {
    store_mat(Rout, R, RP);
    tri_inverse(R, Ri, RP, nullptr);
    store_mat(Tout, Ri, RP);
  }
}

// ---- off the critical path: lagged normaliser of a chain slot ---------------------------
// The chain output of a slot is Q~ = P R_app^{-1} (R_app applied).  The next iteration
// normalises the same slot with T = R_new^{-1}, R_new = chol(Q~^T Q~) R_app (fast path)
// or R_new = R_app (exact path, Q~ already orthonormal).  For products of the last chain
// the applied factor also enters Pi := R_app Pi (the core of eq. mlr_app).
struct SlotArgs {
  const double* g64;       // Gram of Q~ (fast path), or of P when g_is_p (then Q~ = P T_app)
  const float* g32;        // its float copy (nullable)
  int g_is_p;
  const float* R_app[2];   // applied factor, by slot parity (both null: identity)
  const float* T_app[2];   // its inverse (needed when g_is_p)
  const float* L1;         // optional extra left factors: R_app := L2 L1 R_app
  const float* L2;
  float* R_next[2];        // written at index 1 - parity
  float* T_next[2];
  float* Pi;               // RP x RP, nullable
  int pi_mode;             // 0 none, 1 Pi := R_app Pi, 2 Pi := R_app
  int fast;                // compute chol(Gram of Q~)
  int r, RP;
  float alarm_ratio;       // fast path: alarm when the Q~ Cholesky diagonal spread exceeds it
  Ctl* ctl;
};

template <bool WARP>
__global__ void __launch_bounds__(SMALL_THREADS) k_slot(SlotArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort) return;
  extern __shared__ __align__(16) float smf[];
  float (*A)[LD] = reinterpret_cast<float (*)[LD]>(smf);
  float (*B)[LD] = A + kMaxRP;
  float (*C)[LD] = B + kMaxRP;
  float (*D)[LD] = C + kMaxRP;
  float (*E1)[LD] = D + kMaxRP;    // L1
  float (*E2)[LD] = E1 + kMaxRP;   // L2
  float (*TA)[LD] = E2 + kMaxRP;   // T_app
  float (*PI)[LD] = TA + kMaxRP;   // Pi
  const int r = a.r, RP = a.RP;
  const int cur = ctl->slot_parity, nxt = 1 - cur;
  // every input in one phase: the kernel runs beside a product that saturates the
  // memory system, where each dependent round trip costs microseconds
  int nf = 0;
  load_mat_nb(B, a.R_app[cur], RP);                  // B = R_app
  if (a.L1) load_mat_nb(E1, a.L1, RP);
  if (a.L2) load_mat_nb(E2, a.L2, RP);
  if (a.fast && a.g_is_p) load_mat_nb(TA, a.T_app[cur], RP);
  if (a.pi_mode == 1) load_mat_nb(PI, a.Pi, RP);
  if (a.fast) {
    if (a.g32) load_gram32_nb(A, a.g32, r, RP, &nf);
    else load_gram_nb(A, a.g64, r, RP, &nf);
  }
  const int any_nf = __syncthreads_or(nf);
  if (a.L1) mat_mul(E1, B, B, RP, true);             // B = L1 R_app
  if (a.L2) mat_mul(E2, B, B, RP, true);             // B = L2 L1 R_app
  if (a.fast) {
    if (any_nf) {
      if (threadIdx.x == 0) { ctl->nonfinite = 1; ctl->abort = 1; }
      return;
    }
    if (a.g_is_p) {                                  // Gram of Q~ = T^T G T
      mat_mul(A, TA, D, RP, false);                  // D = G T
      for (int e = threadIdx.x; e < kMaxRP * kMaxRP; e += SMALL_THREADS) {
        const int i = e / kMaxRP, j = e % kMaxRP;
        A[i][j] = TA[j][i];                          // A = T^T
      }
      __syncthreads();
      mat_mul(A, D, A, RP, false);                   // A = T^T G T
      for (int e = threadIdx.x; e < kMaxRP * kMaxRP; e += SMALL_THREADS) {
        const int i = e / kMaxRP, j = e % kMaxRP;
        if (i >= r || j >= r) A[i][j] = (i == j) ? 1.f : 0.f;
      }
      __syncthreads();
    }
    __shared__ float dv[kMaxRP];
    robust_chol<WARP>(A, C, D, dv, r, RP, ctl);            // U into C, E into D (scratch)
    for (int e = threadIdx.x; e < kMaxRP * kMaxRP; e += SMALL_THREADS) {   // C = R~, in place
      const int i = e / kMaxRP, c = e % kMaxRP;
      float v = 0.f;
      if (i < RP && c < RP && c >= i) {
        const float si = rsqrtf(dv[i]);
        v = (c == i) ? dv[i] * si : C[i][c] * si;
      }
      C[i][c] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float lo = 3.4e38f, hi = 0.f;
      for (int j = 0; j < r; ++j) { lo = fminf(lo, C[j][j]); hi = fmaxf(hi, C[j][j]); }
      if (!(hi <= a.alarm_ratio * lo)) { ctl->alarm = 1; ctl->abort = 1; }
    }
    mat_mul(C, B, A, RP, true);                      // A = R~ R_app
  } else {
    for (int e = threadIdx.x; e < kMaxRP * kMaxRP; e += SMALL_THREADS) A[e / kMaxRP][e % kMaxRP] = B[e / kMaxRP][e % kMaxRP];
    __syncthreads();
  }
  store_mat(a.R_next[nxt], A, RP);
  tri_inverse(A, C, RP, nullptr);
  store_mat(a.T_next[nxt], C, RP);
  if (a.pi_mode == 2) {
    normalise_into(B, a.Pi, RP, ctl, true);
  } else if (a.pi_mode == 1) {
    mat_mul(B, PI, D, RP, true);                     // D = R_app Pi
    normalise_into(D, a.Pi, RP, ctl, false);
  }
}

// ---- off the critical path: the rank test of Algorithm 1 --------------------------------
// Reading of "rank(A2^T Y1) < r": A2^T Y1 = Y2^T Y2, whose rank is that of Z Q2.  Count
// the pivots of a pivoted Cholesky of (Z Q2)^T (Z Q2) (exact float32 products summed in
// double-float, reduced in float64) above rank_tol^2 of the largest.
__global__ void __launch_bounds__(SMALL_THREADS) k_rank(const double* __restrict__ g64, int r, int RP,
                                                        double rank_tol, Ctl* ctl) {
  if (ctl->abort) return;
  extern __shared__ __align__(16) float smf[];
  double (*Gd)[LD] = reinterpret_cast<double (*)[LD]>(smf);
  __shared__ double dmax0;
  __shared__ int piv, stop, rank;
  const int tid = threadIdx.x;
  for (int e = tid; e < r * r; e += SMALL_THREADS) Gd[e / r][e % r] = g64[(e / r) * RP + e % r];
  if (tid == 0) { stop = 0; rank = r; }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (tid < 32) {
      // pivot: largest remaining diagonal (first index on ties), found by warp 0
      int p = j;
      double best = Gd[j][j];
      for (int i = j + tid; i < r; i += 32)
        if (Gd[i][i] > best || (Gd[i][i] == best && i < p)) { best = Gd[i][i]; p = i; }
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (tid == 0) {
        if (j == 0) dmax0 = best;
        if (!isfinite(best)) {
          ctl->nonfinite = 1;
          ctl->abort = 1;
          stop = 1;
        } else if (!(dmax0 > 0.0) || !(best > rank_tol * rank_tol * dmax0)) {
          rank = j;
          stop = 1;
        }
        piv = p;
      }
    }
    __syncthreads();
    if (stop) break;
    const int p = piv;
    if (p != j) {
      for (int i = tid; i < r; i += SMALL_THREADS) { double t = Gd[j][i]; Gd[j][i] = Gd[p][i]; Gd[p][i] = t; }
      __syncthreads();
      for (int i = tid; i < r; i += SMALL_THREADS) { double t = Gd[i][j]; Gd[i][j] = Gd[i][p]; Gd[i][p] = t; }
      __syncthreads();
    }
    const double invd = 1.0 / Gd[j][j];
    const int w = r - j - 1;
    for (int e = tid; e < w * w; e += SMALL_THREADS) {
      const int aa = j + 1 + e / w, cc = j + 1 + e % w;
      Gd[aa][cc] -= Gd[j][aa] * Gd[j][cc] * invd;       // full symmetric Schur complement
    }
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0 && rank < r && !ctl->nonfinite) {
    ctl->r_eff = rank;
    ctl->rank_drop = 1;
    ctl->abort = 1;
  }
}

// ---- SVD of the core and the singular-value root (eq. mlr_app, reading R4) -------------
// M = Rb Ra Rapp Pi (Rapp optional).  One-sided Jacobi (Hestenes) on W = M V, warm-
// started from the previous iteration's V; column pairs in round-robin order, one warp
// per pair.  V and U are re-orthonormalised with one Newton-Schulz step at the end.
constexpr int SVD_THREADS = 1024;

__device__ void mm_1024(const float (*A)[LD], const float (*B)[LD], float (*C)[LD], int n, bool a_transposed) {
  // C = A B (or A^T B); C must not alias A or B.  The product is bound by shared-memory
  // loads, so 256 of the block's threads each own a 4 x 4 block (rows ty + 16 a, columns
  // tx + 16 b): per K step a warp issues 8 loads for 512 FMAs, against 4 loads for 128 with
  // a 2 x 2 block per thread.  A warp's rows are two values of ty (near-broadcast loads of
  // A); its columns are 16 consecutive ones (conflict-free loads of B).
  const int tid = threadIdx.x;
  if (tid < 256) {
    const int ty = tid >> 4, tx = tid & 15;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 4
    for (int t = 0; t < n; ++t) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = a_transposed ? A[t][ty + 16 * a] : A[ty + 16 * a][t];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = B[t][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = ty + 16 * a, j = tx + 16 * b;
        if (i < n && j < n) C[i][j] = acc[a][b];
      }
  }
  __syncthreads();
}

__device__ void load_1024(float (*D)[LD], const float* src, int RP) {
  for (int e = threadIdx.x; e < RP * RP; e += SVD_THREADS) D[e / RP][e % RP] = src[e];
  __syncthreads();
}

struct SvdArgs2 {
  const float* Ra;
  const float* Rb;
  const float* Rapp[2];    // by slot parity; both null: none
  const float* Pi;         // nullable: identity
  float* Vprev;            // RP x RP, in/out (warm start)
  int r, RP, q;
  float* Um;
  float* Vm;
  float* sigma;
  Ctl* ctl;
  const float* Tl;         // nullable: Um is returned as Tl Um (Tl upper triangular, RP x RP)
};

constexpr float kSvdQuad = 3e-4f;

__global__ void __launch_bounds__(SVD_THREADS) k_svd(SvdArgs2 a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort) return;
  extern __shared__ __align__(16) float smf[];
  float (*X1)[LD] = reinterpret_cast<float (*)[LD]>(smf);
  float (*X2)[LD] = X1 + kMaxRP;
  float (*W)[LD] = X2 + kMaxRP;      // W[row][col] = M V
  float (*V)[LD] = W + kMaxRP;       // V[row][col]
  __shared__ float s[kMaxRP];
  __shared__ int order[kMaxRP];
  __shared__ int rotated;
  __shared__ unsigned s_dmax;        // largest |cos| between a rotated pair in this sweep (float bits)
  __shared__ int s_anyrot;           // some pair was rotated in this call
  __shared__ float s_scale;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, RP = a.RP;
  // M = Rb Ra Rapp Pi
  const float* Rapp = a.Rapp[ctl->slot_parity];
  load_1024(X1, a.Ra, RP);
  if (a.Pi) {
    load_1024(X2, a.Pi, RP);
  } else {
    for (int e = tid; e < RP * RP; e += SVD_THREADS) X2[e / RP][e % RP] = (e / RP == e % RP) ? 1.f : 0.f;
    __syncthreads();
  }
  if (Rapp) {
    load_1024(W, Rapp, RP);
    mm_1024(W, X2, V, RP, false);     // V = Rapp Pi
    mm_1024(X1, V, X2, RP, false);    // X2 = Ra Rapp Pi
  } else {
    mm_1024(X1, X2, V, RP, false);    // V = Ra Pi
    for (int e = tid; e < RP * RP; e += SVD_THREADS) X2[e / RP][e % RP] = V[e / RP][e % RP];
    __syncthreads();
  }
  if (a.Rb) {
    load_1024(X1, a.Rb, RP);
    mm_1024(X1, X2, W, RP, false);    // W = M (unscaled)
  } else {
    for (int e = tid; e < RP * RP; e += SVD_THREADS) W[e / RP][e % RP] = X2[e / RP][e % RP];
    __syncthreads();
  }
  {
    const float mx = block_absmax(W, r);
    if (tid == 0) s_scale = mx > 0.f ? mx : 1.f;
  }
  __syncthreads();
  for (int e = tid; e < RP * RP; e += SVD_THREADS) {
    const int i = e / RP, j = e % RP;
    X2[i][j] = (i < r && j < r) ? W[i][j] / s_scale : 0.f;      // X2 = M / scale
  }
  load_1024(V, a.Vprev, RP);
  for (int e = tid; e < RP * RP; e += SVD_THREADS) {
    const int i = e / RP, j = e % RP;
    if (i >= r || j >= r) V[i][j] = (i == j) ? 1.f : 0.f;       // warm start on the r x r block
  }
  __syncthreads();
  mm_1024(X2, V, W, RP, false);       // W = M V
  // In the steady state the warm start already leaves W's columns orthogonal to the
  // rotation test's resolution, and a sweep would only confirm it (49 dependent rounds at
  // r = 50).  One Gram W^T W (all pairs at once) decides instead: below half the rotation
  // threshold no pair of the sweep could rotate, and the sweeps are skipped.
  mm_1024(W, W, X1, r, true);         // X1 = W^T W
  if (tid == 0) s_dmax = 0u;
  __syncthreads();
  {
    float cmax = 0.f;
    for (int e = tid; e < r * r; e += SVD_THREADS) {
      const int i = e / r, j = e % r;
      if (i < j) {
        const float d = sqrtf(X1[i][i]) * sqrtf(X1[j][j]);
        cmax = fmaxf(cmax, d > 0.f ? fabsf(X1[i][j]) / d : 0.f);
      }
    }
    for (int o = 16; o; o >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    if (lane == 0 && cmax > 0.f) atomicMax(&s_dmax, __float_as_uint(cmax));
  }
  __syncthreads();
  // the same bound as the sweep's rotation test (a pair below it would not be rotated)
  const bool warm_done = __uint_as_float(s_dmax) < 4e-6f;
  if (tid == 0) s_anyrot = 0;
  __syncthreads();

  const int np = (r + 1) & ~1;
  const int npairs = np / 2;
  int sweeps = 0;
  for (; sweeps < 16 && !warm_done; ++sweeps) {
    __syncthreads();                  // every thread has read the previous flag
    if (tid == 0) {
      rotated = 0;
      s_dmax = 0u;
    }
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      if (warp < npairs) {
        int p, q;
        if (warp == 0) { p = np - 1; q = round; }
        else { p = (round + warp) % (np - 1); q = (round - warp + np - 1) % (np - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        if (q < r) {
          float al = 0.f, be = 0.f, ga = 0.f;
          for (int i = lane; i < r; i += 32) {
            const float wp = W[i][p], wq = W[i][q];
            al = fmaf(wp, wp, al);
            be = fmaf(wq, wq, be);
            ga = fmaf(wp, wq, ga);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga += __shfl_xor_sync(0xffffffffu, ga, o);
          }
          // float32 dot products bottom out near sqrt(r) u; 4e-6 keeps a margin above it
          if (fabsf(ga) > 4e-6f * sqrtf(al) * sqrtf(be) && ga != 0.f) {
            const float zeta = (be - al) / (2.f * ga);
            const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
            const float c = 1.f / sqrtf(1.f + t * t);
            const float sn = c * t;
            for (int i = lane; i < r; i += 32) {
              const float wp = W[i][p], wq = W[i][q];
              W[i][p] = c * wp - sn * wq;
              W[i][q] = sn * wp + c * wq;
              const float vp = V[i][p], vq = V[i][q];
              V[i][p] = c * vp - sn * vq;
              V[i][q] = sn * vp + c * vq;
            }
            if (lane == 0) {
              rotated = 1;
              s_anyrot = 1;
              atomicMax(&s_dmax, __float_as_uint(fabsf(ga) / (sqrtf(al) * sqrtf(be))));
            }
          }
        }
      }
      __syncthreads();
    }
    // Cyclic Jacobi converges quadratically: after a sweep whose largest |cos| was below
    // kSvdQuad, the next would see about its square (1e-7), far under the rotation test,
    // and would rotate nothing; it is not run.
    if (!rotated) break;
    if (__uint_as_float(s_dmax) < kSvdQuad) {
      ++sweeps;
      break;
    }
  }
  // Newton-Schulz: V := V (3I - V^T V) / 2 restores orthonormality lost to rounding in
  // the rotations; without any rotation V is the previous call's V, already restored
  __syncthreads();
  if (s_anyrot) {
    mm_1024(V, V, X1, r, true);                     // X1 = V^T V
    for (int e = tid; e < r * r; e += SVD_THREADS) {
      const int i = e / r, j = e % r;
      X1[i][j] = ((i == j) ? 1.5f : 0.f) - 0.5f * X1[i][j];
    }
    __syncthreads();
    mm_1024(V, X1, X2, r, false);                   // X2 = reorthonormalised V
  } else {
    for (int e = tid; e < r * r; e += SVD_THREADS) X2[e / r][e % r] = V[e / r][e % r];
    __syncthreads();
  }
  if (tid < RP) {
    float v = 0.f;
    if (tid < r)
      for (int i = 0; i < r; ++i) v = fmaf(W[i][tid], W[i][tid], v);
    s[tid] = sqrtf(v);
  }
  __syncthreads();
  // descending order of s (ties by column index): column j goes to its rank
  if (tid < RP) {
    int rk = tid;
    if (tid < r) {
      rk = 0;
      for (int i = 0; i < r; ++i) rk += (s[i] > s[tid]) || (s[i] == s[tid] && i < tid);
    }
    order[rk] = tid;
  }
  if (tid == 0) ctl->svd_sweeps = sweeps;
  __syncthreads();
  // U = W diag(1/s), columns in descending order of s; V reordered likewise
  for (int e = tid; e < RP * RP; e += SVD_THREADS) {
    const int i = e / RP, j = e % RP;
    float u = 0.f, v = 0.f;
    if (i < r && j < r) {
      const int c = order[j];
      u = s[c] > 0.f ? W[i][c] / s[c] : 0.f;
      v = X2[i][c];
    }
    X1[i][j] = u;
    V[i][j] = v;
  }
  __syncthreads();
  mm_1024(X1, X1, W, r, true);                      // W = U^T U
  for (int e = tid; e < r * r; e += SVD_THREADS) {
    const int i = e / r, j = e % r;
    W[i][j] = ((i == j) ? 1.5f : 0.f) - 0.5f * W[i][j];
  }
  __syncthreads();
  mm_1024(X1, W, X2, r, false);                     // X2 = reorthonormalised U
  if (a.Tl) {
    load_1024(X1, a.Tl, RP);
    mm_1024(X1, X2, W, r, false);                   // W = Tl U (Tl's padded block does not mix in)
    for (int e = tid; e < r * r; e += SVD_THREADS) X2[e / r][e % r] = W[e / r][e % r];
    __syncthreads();
  }
  for (int e = tid; e < RP * RP; e += SVD_THREADS) {
    const int i = e / RP, j = e % RP;
    const bool in = i < r && j < r;
    a.Um[e] = in ? X2[i][j] : 0.f;
    a.Vm[e] = in ? V[i][j] : 0.f;
    a.Vprev[e] = in ? V[i][j] : (i == j ? 1.f : 0.f);
  }
  if (tid < RP) {
    // float64 only in the two warps that root the singular values (GB300 issues a warp's
    // float64 instruction over many cycles)
    float sv = 0.f;
    if (tid < r) {
      const double inv_e = 1.0 / (double)(2 * a.q + 1);
      const double lsc = (a.Pi ? ctl->m_logscale : 0.0) + log((double)s_scale);
      const float sc = s[order[tid]];
      sv = (sc > 0.f) ? (float)exp((log((double)sc) + lsc) * inv_e) : 0.f;
    }
    a.sigma[tid] = sv;
  }
}

constexpr size_t kSmall4 = 4 * kMaxRP * LD * sizeof(float);
constexpr size_t kSmall8 = 8 * kMaxRP * LD * sizeof(float);

}  // namespace

cudaError_t prepare_small_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_chol<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall4);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall4);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall4);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_slot<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall8);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_slot<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall8);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rank, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall4);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmall4);
  return e;
}

void launch_gram_sum(const void* part, int gram_double, int64_t nblk, int RP, double* out, const Ctl* ctl,
                     cudaStream_t st, float* out32) {
  const int npair = RP * RP;
  // 32 entries per block of 256 threads (8 partials in flight per entry), unless there are
  // few entries and many partials (small r over a tall matrix): then 8 per block of 1024
  if (npair >= 2048 || nblk < 256) {
    const unsigned grid = (unsigned)((npair + 31) / 32);
    if (gram_double)
      k_gram_sum<double, 32, 256><<<grid, 256, 0, st>>>(reinterpret_cast<const double*>(part), nblk, npair, out,
                                                        out32, ctl);
    else
      k_gram_sum<float, 32, 256><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(part), nblk, npair, out, out32,
                                                       ctl);
  } else {
    const unsigned grid = (unsigned)((npair + 7) / 8);
    if (gram_double)
      k_gram_sum<double, 8, 1024><<<grid, 1024, 0, st>>>(reinterpret_cast<const double*>(part), nblk, npair, out,
                                                         out32, ctl);
    else
      k_gram_sum<float, 8, 1024><<<grid, 1024, 0, st>>>(reinterpret_cast<const float*>(part), nblk, npair, out,
                                                        out32, ctl);
  }
}

void launch_chol(const double* g64, int r, int RP, float* R, float* T, Ctl* ctl, cudaStream_t st,
                 float alarm_ratio, bool fp64, const float* g32) {
  if (fp64) k_chol<true, false><<<1, SMALL_THREADS, kSmall4, st>>>(g64, nullptr, r, RP, R, T, alarm_ratio, ctl);
  else if (RP <= 32) k_chol<false, true><<<1, SMALL_THREADS, kSmall4, st>>>(g64, g32, r, RP, R, T, alarm_ratio, ctl);
  else k_chol<false, false><<<1, SMALL_THREADS, kSmall4, st>>>(g64, g32, r, RP, R, T, alarm_ratio, ctl);
}

void launch_slot(const SlotLaunch& l, cudaStream_t st) {
  SlotArgs a;
  a.g64 = l.g64;
  a.g32 = l.g32;
  a.g_is_p = l.g_is_p;
  for (int h = 0; h < 2; ++h) {
    a.R_app[h] = l.R_app[h];
    a.T_app[h] = l.T_app[h];
    a.R_next[h] = l.R_next[h];
    a.T_next[h] = l.T_next[h];
  }
  a.L1 = l.L1;
  a.L2 = l.L2;
  a.Pi = l.Pi;
  a.pi_mode = l.pi_mode;
  a.fast = l.fast;
  a.r = l.r;
  a.RP = l.RP;
  a.alarm_ratio = l.alarm_ratio;
  a.ctl = l.ctl;
  if (l.RP <= 32) k_slot<true><<<1, SMALL_THREADS, kSmall8, st>>>(a);
  else k_slot<false><<<1, SMALL_THREADS, kSmall8, st>>>(a);
}

void launch_rank(const double* g64, int r, int RP, double rank_tol, Ctl* ctl, cudaStream_t st) {
  k_rank<<<1, SMALL_THREADS, kSmall4, st>>>(g64, r, RP, rank_tol, ctl);
}

void launch_svd(const float* Ra, const float* Rb, const float* Rapp0, const float* Rapp1, const float* Pi,
                float* Vprev, int r, int RP, int q, float* Um, float* Vm, float* sigma, Ctl* ctl, cudaStream_t st,
                const float* Tl) {
  SvdArgs2 a{Ra, Rb, {Rapp0, Rapp1}, Pi, Vprev, r, RP, q, Um, Vm, sigma, ctl, Tl};
  k_svd<<<1, SVD_THREADS, kSmall4, st>>>(a);
}

}  // namespace godec
