// Kernels of MSE training (Sec. 4.2.1, Algorithm 4) around the GoDec-BRP L-step: the
// residual R = X - sum_i L^i - S is kept densely; block i works on the rows Omega_i of the
// samples that carry label i.  Each low-rank block L^i lives on its rows only, as factors
// U_i (|Omega_i| x r_i), sigma_i, V_i (p x r_i) once it has been updated (before that it is
// the initial D^{-1} X restricted to Omega_i, eq. msinitial).
#include "godec_internal.cuh"

namespace godec {

namespace {

// value of block i's L^i at (row t of the block, column j): u_t diag(sigma) v_j^T
__device__ __forceinline__ float lr_entry(const float* __restrict__ U, int64_t ldu, const float* __restrict__ sigma,
                                          const float* __restrict__ V, int64_t ldv, int r, int64_t t, int64_t j) {
  float s = 0.f;
  for (int l = 0; l < r; ++l) s = fmaf(U[t * ldu + l] * sigma[l], V[j * ldv + l], s);
  return s;
}

// N (nrows x p, stride ldn) = R[rows] + L^i[rows]: with U null, L^i = X[rows] / D[rows] (the
// initial blocks), else the factored block.
__global__ void k_mse_gather(const float* __restrict__ R, int64_t ldr, const int64_t* __restrict__ rows, int64_t nrows,
                             int64_t p, const float* __restrict__ X, int64_t ldx, const float* __restrict__ invD,
                             const float* __restrict__ U, int64_t ldu, const float* __restrict__ sigma,
                             const float* __restrict__ V, int64_t ldv, int r, float* __restrict__ N, int64_t ldn) {
  const int64_t total = nrows * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / p, j = e % p, i = rows[t];
    const float l = U ? lr_entry(U, ldu, sigma, V, ldv, r, t, j) : X[i * ldx + j] * invD[i];
    N[t * ldn + j] = R[i * ldr + j] + l;
  }
}

// R[rows] = N - L^i[rows] with the new factors of block i.
__global__ void k_mse_scatter(float* __restrict__ R, int64_t ldr, const int64_t* __restrict__ rows, int64_t nrows,
                              int64_t p, const float* __restrict__ N, int64_t ldn, const float* __restrict__ U,
                              int64_t ldu, const float* __restrict__ sigma, const float* __restrict__ V, int64_t ldv,
                              int r) {
  const int64_t total = nrows * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / p, j = e % p;
    R[rows[t] * ldr + j] = N[t * ldn + j] - lr_entry(U, ldu, sigma, V, ldv, r, t, j);
  }
}

// R[idx] += alpha val for COO entries (linear index i p + j; no duplicates).
__global__ void k_sparse_axpy(float* __restrict__ R, int64_t ldr, int64_t p, const int64_t* __restrict__ idx,
                              const float* __restrict__ val, int64_t nnz, float alpha) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx[e] / p, j = idx[e] % p;
    R[i * ldr + j] += alpha * val[e];
  }
}

// out = X - R (rows x p).
__global__ void k_sub(const float* __restrict__ X, int64_t ldx, const float* __restrict__ R, int64_t ldr, int64_t rows,
                      int64_t p, float* __restrict__ out, int64_t ldo) {
  const int64_t total = rows * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / p, j = e % p;
    out[i * ldo + j] = X[i * ldx + j] - R[i * ldr + j];
  }
}

// Initial residual (eq. msinitial): sum_i L^i = X on every row that carries a label (each of
// its D labels holds X / D), so R = 0 there and R = X on unlabelled rows.
__global__ void k_mse_init(const float* __restrict__ X, int64_t ldx, const float* __restrict__ invD, int64_t rows,
                           int64_t p, float* __restrict__ R, int64_t ldr) {
  const int64_t total = rows * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / p, j = e % p;
    R[i * ldr + j] = invD[i] > 0.f ? 0.f : X[i * ldx + j];
  }
}

unsigned grid_for(int64_t total, int nsm) {
  int64_t b = (total + 255) / 256;
  if (b > 16LL * nsm) b = 16LL * nsm;
  return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

void launch_mse_gather(const float* R, int64_t ldr, const int64_t* rows, int64_t nrows, int64_t p, const float* X,
                       int64_t ldx, const float* invD, const float* U, int64_t ldu, const float* sigma, const float* V,
                       int64_t ldv, int r, float* N, int64_t ldn, int nsm, cudaStream_t st) {
  k_mse_gather<<<grid_for(nrows * p, nsm), 256, 0, st>>>(R, ldr, rows, nrows, p, X, ldx, invD, U, ldu, sigma, V, ldv,
                                                         r, N, ldn);
}

void launch_mse_scatter(float* R, int64_t ldr, const int64_t* rows, int64_t nrows, int64_t p, const float* N,
                        int64_t ldn, const float* U, int64_t ldu, const float* sigma, const float* V, int64_t ldv,
                        int r, int nsm, cudaStream_t st) {
  k_mse_scatter<<<grid_for(nrows * p, nsm), 256, 0, st>>>(R, ldr, rows, nrows, p, N, ldn, U, ldu, sigma, V, ldv, r);
}

void launch_sparse_axpy(float* R, int64_t ldr, int64_t p, const int64_t* idx, const float* val, int64_t nnz,
                        float alpha, int nsm, cudaStream_t st) {
  if (nnz > 0) k_sparse_axpy<<<grid_for(nnz, nsm), 256, 0, st>>>(R, ldr, p, idx, val, nnz, alpha);
}

void launch_mse_init(const float* X, int64_t ldx, const float* invD, int64_t rows, int64_t p, float* R, int64_t ldr,
                     int nsm, cudaStream_t st) {
  k_mse_init<<<grid_for(rows * p, nsm), 256, 0, st>>>(X, ldx, invD, rows, p, R, ldr);
}

void launch_sub(const float* X, int64_t ldx, const float* R, int64_t ldr, int64_t rows, int64_t p, float* out,
                int64_t ldo, int nsm, cudaStream_t st) {
  k_sub<<<grid_for(rows * p, nsm), 256, 0, st>>>(X, ldx, R, ldr, rows, p, out, ldo);
}

}  // namespace godec
