// Kernels of GreBsmo (Sec. 3.2.1, Algorithm 2 with the updates of eq. GreBsmoA) that the
// GoDec-BRP path does not already have.  The streaming products, CholeskyQR, the
// tensor-core residual pass and the sparse update of X - S are shared with GoDec.
//
// S-step (eq. softt): S = S_lambda(X - U V).  Only the entries with |R| > lambda are
// nonzero, so the residual pass runs in its candidate mode with the threshold key of
// lambda + 1 ulp (no selection follows: every candidate is in the support) and the emit
// writes S = R - lambda sgn R.  The objective then needs no second pass:
// ||X - U V - S||^2 = (sum of R^2 over |R| <= lambda) + |supp S| lambda^2.
#include "godec_internal.cuh"

namespace godec {

namespace {

// Plan of a GreBsmo S-step, after the per-iteration reset: one candidate pass at `guess`.
__global__ void k_soft_plan(Ctl* ctl, unsigned guess) {
  ctl->plan[0] = PASS_CAND;
  ctl->plan[1] = PASS_NONE;
  ctl->plan[2] = PASS_NONE;
  ctl->guess[0] = guess;
  ctl->cand_count = 0ull;
  ctl->sumsq_noncand = 0.0;
}

constexpr int SOFT_THREADS = 256;

__global__ void __launch_bounds__(SOFT_THREADS) k_emit_soft(SoftEmitArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort) return;
  const unsigned long long cnt = ctl->cand_count;
  if (cnt > a.cand_cap || cnt > (unsigned long long)a.s_cap) {
    // the support outgrew the buffers: the host grows them and redoes the S-step
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->need_bigger_cand = 1;
      ctl->abort = 1;
    }
    return;
  }
  const int nb = ctl->cur ^ 1;
  long long* Sidx = a.S_idx[nb];
  float* Sval = a.S_val[nb];
  unsigned* bits = a.sbits ? a.sbits + (size_t)nb * (size_t)a.sbits_words : nullptr;   // clear until now
  for (unsigned long long e = (unsigned long long)blockIdx.x * SOFT_THREADS + threadIdx.x; e < cnt;
       e += (unsigned long long)gridDim.x * SOFT_THREADS) {
    const long long idx = a.cand_idx[e];
    const float v = a.cand_val[e];
    Sidx[e] = idx;
    Sval[e] = v - copysignf(a.lambda, v);   // sgn(R) (|R| - lambda), |R| > lambda
    if (bits) atomicOr(&bits[idx >> 5], 1u << (idx & 31));
  }
  __threadfence();
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&ctl->done_ctas2, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  const double lam = (double)a.lambda;
  const double obj = atomicAdd(&ctl->sumsq_noncand, 0.0) + (double)cnt * lam * lam;
  ctl->obj = obj;
  ctl->rel_err = ctl->normX2 > 0.0 ? obj / ctl->normX2 : 0.0;
  ctl->nnz_prev = ctl->nnz_cur;
  ctl->nnz_cur = (long long)cnt;
  ctl->cur = nb;
  ctl->iter += 1;
  ctl->last_passes = 1;
  ctl->done_ctas2 = 0u;
}

// sigma_l = sqrt(G_ll) (the column norms of W, from its Gram) for l < r, else 0;
// Vh = W diag(1 / sigma) (unit columns; zero beyond r).
__global__ void k_colnorm(const float* __restrict__ W, const double* __restrict__ g64, int64_t n, int RP, int r,
                          float* __restrict__ Vh, float* __restrict__ sigma, const int* skip) {
  if (block_skip(skip)) return;
  // the column norms and their inverses once per block, in float32 (float64 arithmetic on
  // every element would queue on GB300's slow float64 pipe)
  __shared__ float inv[kMaxRP];
  if (threadIdx.x < RP) {
    const int l = threadIdx.x;
    const float s = l < r ? sqrtf(fmaxf((float)g64[(size_t)l * RP + l], 0.f)) : 0.f;
    inv[l] = s > 0.f ? 1.f / s : 0.f;
    if (blockIdx.x == 0) sigma[l] = s;
  }
  __syncthreads();
  const int64_t total = n * RP;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Vh[e] = W[e] * inv[e % RP];
}

// out (r x r, stored as float64, row-major) = A B, or (A B)^T with trans, then row i times
// rowscale[i]; A, B float32 with stride ld, accumulated in float32.
__global__ void k_rmul(const float* __restrict__ A, const float* __restrict__ B, int ld, int r, double* __restrict__ out,
                       int trans, const float* __restrict__ rowscale, const int* skip) {
  if (block_skip(skip)) return;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e % r;
    float s = 0.f;   // float32 accumulation: the factors are float32 and r <= 64
    for (int k = 0; k < r; ++k) s = fmaf(A[i * ld + k], B[k * ld + j], s);
    const int oi = trans ? j : i, oj = trans ? i : j;
    out[oi * r + oj] = rowscale ? (double)(s * rowscale[oi]) : (double)s;
  }
}

// LinGoDec's W = U_L diag(sigma) (Rf^{-1} Vr)^T: out (d x r, float64, row-major) =
// T1 T2 Vr diag(sigma) with T1, T2 the float32 inverses of F's two CholeskyQR factors
// (stride ld, upper triangular, d x d) and Vr (d x r, float64, stride r).
__global__ void k_lingo_g(const float* __restrict__ T1, const float* __restrict__ T2, int ld,
                          const double* __restrict__ Vr, const float* __restrict__ sigma, int d, int r,
                          double* __restrict__ out) {
  __shared__ double tmp[kMaxRP * kMaxRP];
  for (int e = threadIdx.x; e < d * r; e += blockDim.x) {   // tmp = T2 Vr diag(sigma)
    const int i = e / r, j = e % r;
    double s = 0.0;
    for (int k = i; k < d; ++k) s += (double)T2[i * ld + k] * Vr[k * r + j];
    tmp[e] = s * (double)sigma[j];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < d * r; e += blockDim.x) {   // out = T1 tmp
    const int i = e / r, j = e % r;
    double s = 0.0;
    for (int k = i; k < d; ++k) s += (double)T1[i * ld + k] * tmp[k * r + j];
    out[e] = s;
  }
}

}  // namespace

void launch_lingo_g(const float* T1, const float* T2, int ld, const double* Vr, const float* sigma, int d, int r,
                    double* out, cudaStream_t st) {
  k_lingo_g<<<1, 256, 0, st>>>(T1, T2, ld, Vr, sigma, d, r, out);
}

void launch_soft_plan(Ctl* ctl, unsigned guess, cudaStream_t st) { k_soft_plan<<<1, 1, 0, st>>>(ctl, guess); }

void launch_emit_soft(const SoftEmitArgs& a, int nsm, cudaStream_t st) {
  k_emit_soft<<<(unsigned)(2 * nsm), SOFT_THREADS, 0, st>>>(a);
}

void launch_colnorm(const float* W, const double* g64, int64_t n, int RP, int r, float* Vh, float* sigma, int nsm,
                    cudaStream_t st, const int* skip) {
  int64_t blocks = (n * RP + 255) / 256;
  if (blocks > 8LL * nsm) blocks = 8LL * nsm;
  k_colnorm<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(W, g64, n, RP, r, Vh, sigma, skip);
}

void launch_rmul(const float* A, const float* B, int ld, int r, double* out, int trans, const float* rowscale,
                 cudaStream_t st, const int* skip) {
  k_rmul<<<1, 256, 0, st>>>(A, B, ld, r, out, trans, rowscale, skip);
}

}  // namespace godec
