// r x r kernels of the L-step, one thread block each.
//
//  * k_chol : Gram matrix of a tall factor (sum of 64-row partials in a fixed
//    order) -> Cholesky R with G = R^T R -> R^{-1}; optionally accumulates the
//    core M := R M of the last power chain (eq. mlr_app: with Q2 = orth(Y2),
//    L~ Q2 = Q1 R_{2q} ... R_0, and R1 (A2^T Y1)^{-1} R2^T equals that product).
//    With rank_test set it first runs a pivoted Cholesky in float64 on an
//    exactly accumulated Gram and counts pivots above rank_tol^2 of the
//    largest: the numerical rank of Z Q2, i.e. of A2^T Y1 (Algorithm 1 line 7).
//  * k_svd_root : one-sided Jacobi SVD of M, then sigma^(1/(2q+1)) (eq.
//    mlr_app, singular-value root).
//
// GB300 runs float64 at about 2 FMA per clock per SM, so only the rank test
// (about r^3/6 float64 FMAs) uses it; everything else here is float32.
#include <math.h>

#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int CHOL_THREADS = 256;
constexpr size_t kCholSmem = 3 * kMaxRP * (kMaxRP + 1) * sizeof(float);

// Sum the Gram partials of all 64-row blocks in float64, one entry per thread,
// spread over many blocks (a single block would be bound by load latency).
template <typename T>
__global__ void k_gram_sum(const T* __restrict__ part, int64_t nblk, int npair, double* __restrict__ out,
                           const Ctl* ctl) {
  if (ctl && ctl->abort) return;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npair) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t b = 0;
  for (; b + 4 <= nblk; b += 4) {
    s0 += (double)part[(b + 0) * npair + e];
    s1 += (double)part[(b + 1) * npair + e];
    s2 += (double)part[(b + 2) * npair + e];
    s3 += (double)part[(b + 3) * npair + e];
  }
  for (; b < nblk; ++b) s0 += (double)part[b * npair + e];
  out[e] = (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(CHOL_THREADS)
k_chol(CholArgs a, const double* __restrict__ gram64) {
  Ctl* ctl = a.ctl;
  if (ctl->abort) return;
  // G, then R and R^{-1}; the float64 rank-test matrix aliases R and R^{-1}.
  extern __shared__ __align__(16) unsigned char chol_smem[];
  typedef float Row[kMaxRP + 1];
  typedef double RowD[kMaxRP + 1];
  Row* G = reinterpret_cast<Row*>(chol_smem);
  Row* R = G + kMaxRP;
  Row* Ri = R + kMaxRP;
  RowD* Gd = reinterpret_cast<RowD*>(R);
  __shared__ int s_rank;
  const int tid = threadIdx.x;
  const int r = a.r, RP = a.RP;
  const int npair = RP * RP;

  // ---- Gram matrix (reduced over row blocks in float64 by k_gram_sum) ----------------
  for (int e = tid; e < npair; e += CHOL_THREADS) {
    int i = e / RP, j = e % RP;
    double v = gram64[e];
    if (a.rank_test) Gd[i][j] = v;
    G[i][j] = (float)v;
  }
  __syncthreads();

  // ---- non-finite Gram: X - S holds NaN/Inf ---------------------------------------------
  {
    __shared__ int s_nf;
    if (tid == 0) s_nf = 0;
    __syncthreads();
    for (int e = tid; e < npair; e += CHOL_THREADS)
      if (!isfinite(G[e / RP][e % RP])) s_nf = 1;
    __syncthreads();
    if (s_nf) {
      if (tid == 0) {
        ctl->nonfinite = 1;
        ctl->abort = 1;
      }
      return;
    }
  }

  // ---- numerical rank by pivoted Cholesky in float64 ------------------------------------
  if (a.rank_test) {
    if (tid == 0) {
      // one thread: r is at most 64 and the update is done by the block below
      s_rank = r;
    }
    __syncthreads();
    __shared__ double dmax0;
    __shared__ int piv;
    __shared__ int stop;
    if (tid == 0) stop = 0;
    for (int j = 0; j < r; ++j) {
      if (tid == 0) {
        int p = j;
        double best = Gd[j][j];
        for (int i = j + 1; i < r; ++i)
          if (Gd[i][i] > best) { best = Gd[i][i]; p = i; }
        if (j == 0) dmax0 = best;
        if (!(best > a.rank_tol * a.rank_tol * dmax0) || !(dmax0 > 0.0)) {
          s_rank = j;
          stop = 1;
        }
        piv = p;
      }
      __syncthreads();
      if (stop) break;
      const int p = piv;
      if (p != j) {   // symmetric swap of row/column j and p
        for (int i = tid; i < r; i += CHOL_THREADS) {
          double t = Gd[j][i]; Gd[j][i] = Gd[p][i]; Gd[p][i] = t;
        }
        __syncthreads();
        for (int i = tid; i < r; i += CHOL_THREADS) {
          double t = Gd[i][j]; Gd[i][j] = Gd[i][p]; Gd[i][p] = t;
        }
        __syncthreads();
      }
      const double d = sqrt(Gd[j][j]);
      __syncthreads();
      for (int c = j + 1 + tid; c < r; c += CHOL_THREADS) Gd[j][c] /= d;
      __syncthreads();
      const int w = r - j - 1;
      for (int e = tid; e < w * w; e += CHOL_THREADS) {
        int aa = j + 1 + e / w, cc = j + 1 + e % w;
        if (cc >= aa) Gd[aa][cc] -= Gd[j][aa] * Gd[j][cc];
      }
      __syncthreads();
      for (int e = tid; e < w * w; e += CHOL_THREADS) {
        int aa = j + 1 + e / w, cc = j + 1 + e % w;
        if (cc < aa) Gd[aa][cc] = Gd[cc][aa];
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_rank < r) {
      if (tid == 0) {
        ctl->r_eff = s_rank;
        ctl->rank_drop = 1;
        ctl->abort = 1;
      }
      return;
    }
  }

  // ---- Cholesky G = R^T R (float32, right-looking) -------------------------------------
  // Pivots below 1e-6 of the largest diagonal mean the factor is numerically rank
  // deficient (noise columns of a power chain whose Z has rank < r); the factorisation
  // is then redone on G + shift*I (shifted CholeskyQR), which keeps Q bounded until
  // the rank test of the last chain lowers r.
  __shared__ float s_d;
  __shared__ float s_gmax;
  __shared__ int s_bad;
  for (int e = tid; e < npair; e += CHOL_THREADS) {
    int i = e / RP, j = e % RP;
    if (i >= r || j >= r) G[i][j] = (i == j) ? 1.f : 0.f;   // padded columns: identity
    Ri[i][j] = G[i][j];                                      // keep a copy for a retry
  }
  __syncthreads();
  if (tid == 0) {
    float gm = 0.f;
    for (int j = 0; j < r; ++j) gm = fmaxf(gm, G[j][j]);
    s_gmax = gm;
    if (!isfinite(gm)) ctl->nonfinite = 1;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      for (int e = tid; e < npair; e += CHOL_THREADS) {
        int i = e / RP, j = e % RP;
        G[i][j] = Ri[i][j] + ((i == j && i < r) ? 1e-5f * s_gmax : 0.f);
      }
    }
    for (int e = tid; e < npair; e += CHOL_THREADS) R[e / RP][e % RP] = 0.f;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    const float thr = 1e-6f * s_gmax;
    for (int j = 0; j < RP; ++j) {
      // Every thread reads pivot j itself, so row j of R and the trailing update
      // need no barrier between them; one barrier per column.
      float d = G[j][j];
      if (!(d > thr) && j < r) {
        if (tid == 0) s_bad = 1;
        if (!(d > 0.f)) d = thr + 1e-30f;
      }
      const float sq = sqrtf(d);
      const float invd = 1.f / d;
      for (int c = j + tid; c < RP; c += CHOL_THREADS) R[j][c] = (c == j) ? sq : G[j][c] / sq;
      const int w = RP - j - 1;
      for (int e = tid; e < w * w; e += CHOL_THREADS) {
        int aa = j + 1 + e / w, cc = j + 1 + e % w;
        if (cc >= aa) G[aa][cc] -= G[j][aa] * G[j][cc] * invd;
      }
      __syncthreads();
    }
    if (!s_bad) break;
    if (tid == 0) ctl->chol_shifts += 1;
    __syncthreads();
  }

  // ---- R^{-1}: row i of the inverse from rows below (all columns in parallel) ----------
  for (int e = tid; e < npair; e += CHOL_THREADS) Ri[e / RP][e % RP] = 0.f;
  __syncthreads();
  for (int i = RP - 1; i >= 0; --i) {
    for (int c = i + tid; c < RP; c += CHOL_THREADS) {
      float v;
      if (c == i) {
        v = 1.f / R[i][i];
      } else {
        float s = 0.f;
        for (int j = i + 1; j <= c; ++j) s = fmaf(R[i][j], Ri[j][c], s);
        v = -s / R[i][i];
      }
      Ri[i][c] = v;
    }
    __syncthreads();
  }
  for (int e = tid; e < npair; e += CHOL_THREADS) {
    int i = e / RP, j = e % RP;
    a.R[e] = R[i][j];
    a.Rinv[e] = Ri[i][j];
  }

  // ---- core of the last chain: M := R M ------------------------------------------------
  // M grows like sigma^(2q+1); it is kept divided by its scale, with log(scale) in
  // float64 in the control block, so float32 never overflows.
  if (a.accumulate) {
    __shared__ float s_scale;
    __syncthreads();
    if (tid == 0) {
      float mx = 0.f;
      for (int i = 0; i < RP; ++i)
        for (int j = i; j < RP; ++j) mx = fmaxf(mx, fabsf(R[i][j]));
      s_scale = mx > 0.f ? mx : 1.f;
      ctl->m_logscale = (a.accumulate == 2 ? 0.0 : ctl->m_logscale) + log((double)s_scale);
    }
    __syncthreads();
    const float inv = 1.f / s_scale;
    if (a.accumulate == 2) {
      for (int e = tid; e < npair; e += CHOL_THREADS) a.M[e] = R[e / RP][e % RP] * inv;
    } else {
      // G is free now: hold the old M there.
      for (int e = tid; e < npair; e += CHOL_THREADS) G[e / RP][e % RP] = a.M[e];
      __syncthreads();
      for (int e = tid; e < npair; e += CHOL_THREADS) {
        int i = e / RP, j = e % RP;
        float acc = 0.f;
        for (int t = i; t < RP; ++t) acc = fmaf(R[i][t] * inv, G[t][j], acc);
        a.M[e] = acc;
      }
    }
  }
}

// ----------------------------------------------------------------------------------
// One-sided Jacobi SVD (Hestenes) of M, parallel round-robin ordering: one warp per
// column pair.  M = W V^T with W = U diag(s).
// ----------------------------------------------------------------------------------
constexpr int SVD_THREADS = 1024;

__global__ void __launch_bounds__(SVD_THREADS)
k_svd_root(SvdArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort) return;
  __shared__ float W[kMaxRP][kMaxRP + 1];   // W[col][row]
  __shared__ float V[kMaxRP][kMaxRP + 1];   // V[col][row]
  __shared__ float s[kMaxRP];
  __shared__ int order[kMaxRP];
  __shared__ int rotated;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, RP = a.RP;
  for (int e = tid; e < RP * RP; e += SVD_THREADS) {
    int i = e / RP, j = e % RP;            // M[i][j]
    W[j][i] = (i < r && j < r) ? a.M[e] : 0.f;
    V[j][i] = (i == j) ? 1.f : 0.f;
  }
  const int np = (r + 1) & ~1;             // even number of players
  const int npairs = np / 2;
  int sweeps = 0;
  for (; sweeps < 40; ++sweeps) {
    __syncthreads();          // every thread has read the previous sweep's flag
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      if (warp < npairs) {
        int p, q;
        if (warp == 0) {
          p = np - 1;
          q = round;
        } else {
          p = (round + warp) % (np - 1);
          q = (round - warp + np - 1) % (np - 1);
        }
        if (p > q) { int t = p; p = q; q = t; }
        if (q < r) {
          float al = 0.f, be = 0.f, ga = 0.f;
          for (int i = lane; i < r; i += 32) {
            float wp = W[p][i], wq = W[q][i];
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
          if (fabsf(ga) > 1e-6f * sqrtf(al) * sqrtf(be) && ga != 0.f) {
            float zeta = (be - al) / (2.f * ga);
            float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
            float c = rsqrtf(1.f + t * t);
            float sn = c * t;
            for (int i = lane; i < r; i += 32) {
              float wp = W[p][i], wq = W[q][i];
              W[p][i] = c * wp - sn * wq;
              W[q][i] = sn * wp + c * wq;
              float vp = V[p][i], vq = V[q][i];
              V[p][i] = c * vp - sn * vq;
              V[q][i] = sn * vp + c * vq;
            }
            if (lane == 0) rotated = 1;
          }
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
  }
  // singular values and ordering
  if (tid < RP) {
    float v = 0.f;
    if (tid < r)
      for (int i = 0; i < r; ++i) v = fmaf(W[tid][i], W[tid][i], v);
    s[tid] = sqrtf(v);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < RP; ++j) order[j] = j;
    for (int j = 0; j < r; ++j) {          // selection sort, descending
      int b = j;
      for (int i = j + 1; i < r; ++i)
        if (s[order[i]] > s[order[b]]) b = i;
      int t = order[j]; order[j] = order[b]; order[b] = t;
    }
    ctl->svd_sweeps = sweeps;
  }
  __syncthreads();
  const double inv_e = 1.0 / (double)(2 * a.q + 1);
  const double lsc = ctl->m_logscale;
  for (int e = tid; e < RP * RP; e += SVD_THREADS) {
    int i = e / RP, j = e % RP;            // output [row i][col j]
    float u = 0.f, v = 0.f;
    if (j < r) {
      int c = order[j];
      float sc = s[c];
      u = (sc > 0.f && i < r) ? W[c][i] / sc : 0.f;
      v = (i < r) ? V[c][i] : 0.f;
    }
    a.Um[e] = u;
    a.Vm[e] = v;
  }
  if (tid < RP) {
    float sv = 0.f;
    if (tid < r) {
      float sc = s[order[tid]];
      sv = (sc > 0.f) ? (float)exp((log((double)sc) + lsc) * inv_e) : 0.f;
    }
    a.sigma[tid] = sv;
  }
}

}  // namespace

void launch_chol(const CholArgs& a, cudaStream_t st) {
  // the reduced Gram goes after the partials in the same buffer (no overlap for
  // float or double partials: it starts at byte 8 * nblk * npair)
  const int npair = a.RP * a.RP;
  double* out = reinterpret_cast<double*>(const_cast<void*>(a.gram_part)) + a.nblk * npair;
  const unsigned grid = (unsigned)((npair + 127) / 128);
  if (a.gram_double)
    k_gram_sum<double><<<grid, 128, 0, st>>>(reinterpret_cast<const double*>(a.gram_part), a.nblk, npair, out, a.ctl);
  else
    k_gram_sum<float><<<grid, 128, 0, st>>>(reinterpret_cast<const float*>(a.gram_part), a.nblk, npair, out, a.ctl);
  k_chol<<<1, CHOL_THREADS, kCholSmem, st>>>(a, out);
}

cudaError_t prepare_small_kernels() {
  return cudaFuncSetAttribute(k_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmem);
}

void launch_svd_root(const SvdArgs& a, cudaStream_t st) {
  k_svd_root<<<1, SVD_THREADS, 0, st>>>(a);
}

}  // namespace godec
