// Kernels of the precision form's float32 correction (reading of the paper's error
// control for the rounded chain; the oracle is tangent_refine): the 16-bit copies of the
// working matrix, the 2r x 2r core of the tangent-space re-truncation and its SVD.
#include <cuda_fp16.h>

#include "godec_internal.cuh"

namespace godec {

namespace {

// dst (rows x cols, float16, row stride ldd) = src (float32, row stride lds), rounded to
// nearest (src holds (X - S) s_Z, inside the float16 range).
__global__ void k_to_half(const float* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                          __half* __restrict__ dst, int64_t ldd) {
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x)
    for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) dst[i * ldd + j] = __float2half_rn(src[i * lds + j]);
}

// W (rows x ld) = [P | Q | 0]: P and Q rows x r (row stride ldp), zero columns 2r..ld-1.
__global__ void k_concat2(const float* __restrict__ P, const float* __restrict__ Q, int64_t ldp, int r, int64_t rows,
                          float* __restrict__ W, int ld, const int* skip) {
  if (block_skip(skip)) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * ld) return;
  const int64_t i = e / ld;
  const int j = (int)(e % ld);
  W[e] = j < r ? P[i * ldp + j] : (j < 2 * r ? Q[i * ldp + j - r] : 0.f);
}

// core = Ra K Rb^T, n2 = 2r:  Ra = Ra2 Ra1 and Rb = Rb2 Rb1 (upper, stride ld), K = [[-C, I],
// [I, 0]] with C (r x r, float64, stride r).  One block; the result in float64 (stride n2).
__global__ void k_refine_core(const float* __restrict__ Ra1, const float* __restrict__ Ra2,
                              const float* __restrict__ Rb1, const float* __restrict__ Rb2, int ld,
                              const double* __restrict__ C, int r, double* __restrict__ core, const int* skip) {
  if (block_skip(skip)) return;
  extern __shared__ double smd[];   // Ra, Rb, K: 3 x 64 x 65 doubles (dynamic)
  double (*Ra)[kMaxRP + 1] = reinterpret_cast<double (*)[kMaxRP + 1]>(smd);
  double (*Rb)[kMaxRP + 1] = Ra + kMaxRP;
  double (*Km)[kMaxRP + 1] = Rb + kMaxRP;
  const int n2 = 2 * r, tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n2 * n2; e += nt) {
    const int i = e / n2, j = e % n2;
    double sa = 0.0, sb = 0.0;
    for (int k = 0; k < n2; ++k) {
      sa += (double)Ra2[i * ld + k] * (double)Ra1[k * ld + j];
      sb += (double)Rb2[i * ld + k] * (double)Rb1[k * ld + j];
    }
    Ra[i][j] = sa;
    Rb[i][j] = sb;
    double kv = 0.0;
    if (i < r && j < r) kv = -C[i * r + j];
    else if (i < r && j == i + r) kv = 1.0;
    else if (i >= r && j == i - r) kv = 1.0;
    Km[i][j] = kv;
  }
  __syncthreads();
  // core[i][j] = sum_p Ra[i][p] sum_q K[p][q] Rb[j][q]
  for (int e = tid; e < n2 * n2; e += nt) {
    const int i = e / n2, j = e % n2;
    double s = 0.0;
    for (int p = 0; p < n2; ++p) {
      double t = 0.0;
      for (int q = 0; q < n2; ++q) t += Km[p][q] * Rb[j][q];
      s += Ra[i][p] * t;
    }
    core[i * n2 + j] = s;
  }
}

constexpr double kJacobiTol = 1e-14;

// SVD of an n x n float64 matrix (n <= 64) by one-sided Jacobi (Hestenes): columns of
// W = A V are rotated pairwise until orthogonal.  Round-robin ordering: each round the
// n/2 disjoint pairs go to one warp each (rows lane and lane + 32), one barrier per round.
// Cyclic Jacobi converges quadratically, so a sweep whose largest |cos| between rotated
// columns was below kJacobiQuad ends the iteration (the next would be near kJacobiTol).
// Outputs the r leading singular triplets, descending: U[:, :r] (n x r, float64, stride
// r), sigma[:r] (float32), V[:, :r] (n x r, stride r).  Launched with 32 ceil(n/2) threads.
constexpr double kJacobiQuad = 1e-7;
// float32: a length-64 dot product bottoms out near sqrt(64) 2^-24, so pairs are rotated
// down to 2e-6; the sweeps go on until one rotates nothing (no early stop on quadratic
// convergence: the singular vectors feed least-squares factors whose error reaches S)
constexpr float kJacobiTolF = 2e-6f;
constexpr double kJacobiQuadF = 0.0;

// T = double, or float for the larger cores of the subspace iterations (GB300 issues a
// warp's float64 instruction over many cycles: a float64 sweep over 58 columns costs
// hundreds of microseconds); float32 rotates down to kJacobiTolF.
template <typename T>
__global__ void __launch_bounds__(1024) k_svd_small(const double* __restrict__ A, int n, int r, double* __restrict__ Uo,
                                                    float* __restrict__ sigma, double* __restrict__ Vo,
                                                    const int* skip) {
  if (block_skip(skip)) return;
  extern __shared__ double smd[];   // W, V: 2 x 64 x 65 values (dynamic)
  T (*W)[kMaxRP + 1] = reinterpret_cast<T (*)[kMaxRP + 1]>(smd);
  T (*V)[kMaxRP + 1] = W + kMaxRP;
  __shared__ T nrm[kMaxRP];
  __shared__ int order[kMaxRP];
  __shared__ int s_rot;
  __shared__ unsigned long long s_dmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    W[i][j] = (T)A[e];
    V[i][j] = (i == j) ? (T)1 : (T)0;
  }
  const int np = (n + 1) & ~1, npairs = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    __syncthreads();
    if (tid == 0) {
      s_rot = 0;
      s_dmax = 0ull;
    }
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
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q < n) {
          T a = 0, b = 0, g = 0;
          for (int i = lane; i < n; i += 32) {
            const T wp = W[i][p], wq = W[i][q];
            a += wp * wp;
            b += wq * wq;
            g += wp * wq;
          }
          for (int o = 16; o; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            g += __shfl_xor_sync(0xffffffffu, g, o);
          }
          // rotate unless the pair is orthogonal to the rounding level of a length-64 dot
          // product in float64 (a tighter test never ends: rounding keeps |g| near it)
          const T tol = sizeof(T) == 8 ? (T)kJacobiTol : (T)kJacobiTolF;
          if (fabs(g) > tol * sqrt(a * b) && g != (T)0) {
            const T zeta = (b - a) / (2 * g);
            const T t = (zeta >= 0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt(1 + zeta * zeta));
            const T cs = 1 / sqrt(1 + t * t), sn = cs * t;
            for (int i = lane; i < n; i += 32) {
              const T wp = W[i][p], wq = W[i][q], vp = V[i][p], vq = V[i][q];
              W[i][p] = cs * wp - sn * wq;
              W[i][q] = sn * wp + cs * wq;
              V[i][p] = cs * vp - sn * vq;
              V[i][q] = sn * vp + cs * vq;
            }
            if (lane == 0) {
              s_rot = 1;
              atomicMax(&s_dmax, (unsigned long long)__double_as_longlong((double)(fabs(g) / sqrt(a * b))));
            }
          }
        }
      }
      __syncthreads();
    }
    if (!s_rot || __longlong_as_double((long long)s_dmax) < (sizeof(T) == 8 ? kJacobiQuad : kJacobiQuadF)) break;
  }
  // column norms, descending order
  for (int i = tid; i < n; i += nt) {
    T sm = 0;
    for (int k = 0; k < n; ++k) sm += W[k][i] * W[k][i];
    nrm[i] = sqrt(sm);
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    int rank = 0;
    for (int k = 0; k < n; ++k) rank += (nrm[k] > nrm[i]) || (nrm[k] == nrm[i] && k < i);
    order[rank] = i;
  }
  __syncthreads();
  for (int e = tid; e < n * r; e += nt) {
    const int i = e / r, j = e % r;
    const int col = order[j];
    const double sv = (double)nrm[col];
    Uo[i * r + j] = sv > 0.0 ? (double)W[i][col] / sv : 0.0;
    Vo[i * r + j] = (double)V[i][col];
  }
  for (int j = tid; j < r; j += nt) sigma[j] = (float)nrm[order[j]];
}

}  // namespace

void launch_to_half(const float* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd, int nsm,
                     cudaStream_t st) {
  int64_t grid = 4LL * nsm;
  if (grid > rows) grid = rows;
  if (grid > 0) k_to_half<<<(unsigned)grid, 256, 0, st>>>(src, rows, cols, lds, static_cast<__half*>(dst), ldd);
}

void launch_concat2(const float* P, const float* Q, int64_t ldp, int r, int64_t rows, float* W, int ld,
                    cudaStream_t st, const int* skip) {
  const int64_t total = rows * ld;
  if (total > 0) k_concat2<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(P, Q, ldp, r, rows, W, ld, skip);
}

constexpr size_t kCoreSmem = 3 * kMaxRP * (kMaxRP + 1) * sizeof(double);
constexpr size_t kSvdSmem = 2 * kMaxRP * (kMaxRP + 1) * sizeof(double);

cudaError_t prepare_refine_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_refine_core, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoreSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_svd_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSvdSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_svd_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSvdSmem);
  return e;
}

void launch_refine_core(const float* Ra1, const float* Ra2, const float* Rb1, const float* Rb2, int ld,
                        const double* C, int r, double* core, cudaStream_t st, const int* skip) {
  k_refine_core<<<1, 256, kCoreSmem, st>>>(Ra1, Ra2, Rb1, Rb2, ld, C, r, core, skip);
}

void launch_svd_small(const double* A, int n, int r, double* U, float* sigma, double* V, cudaStream_t st,
                      const int* skip, bool f32) {
  if (f32) k_svd_small<float><<<1, 32 * ((n + 1) / 2), kSvdSmem, st>>>(A, n, r, U, sigma, V, skip);
  else k_svd_small<double><<<1, 32 * ((n + 1) / 2), kSvdSmem, st>>>(A, n, r, U, sigma, V, skip);
}

}  // namespace godec
