// Kernels of the differentiated form (q = 0, supports frozen): tall x small products,
// cross Grams A^T B of tall matrices, sparse (COO) times tall products, low-rank values
// at COO positions, and the dense accumulation of low-rank terms into dX.  The streaming
// products with the iterate Z_t run on the tensor-core kernel of the forward pass.
#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int BW_THREADS = 256;

// C = A^T B over a fixed row partition: block g adds rows [g R / G, (g+1) R / G) into
// part[g] (a x b, float64), 32-row chunks staged in shared memory (only the a and b
// columns in use); a, b <= 64.  Each thread owns entries tid + 256 k of a x b.
__global__ void __launch_bounds__(BW_THREADS)
k_cross_part(const float* __restrict__ A, int64_t lda, int a, const float* __restrict__ B, int64_t ldb, int b,
             int64_t rows, double* __restrict__ part, const int* skip) {
  if (block_skip(skip)) return;
  constexpr int CH = 32;
  __shared__ float sA[CH][kMaxRP + 1], sB[CH][kMaxRP + 1];
  const int tid = threadIdx.x, G = gridDim.x, g = blockIdx.x;
  const int64_t r0 = (int64_t)g * rows / G, r1 = (int64_t)(g + 1) * rows / G;
  const int ne = a * b;
  double acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  for (int64_t c0 = r0; c0 < r1; c0 += CH) {
    const int nr = (int)(r1 - c0 < CH ? r1 - c0 : CH);
    __syncthreads();
    for (int e = tid; e < nr * a; e += BW_THREADS) sA[e / a][e % a] = A[(c0 + e / a) * lda + e % a];
    for (int e = tid; e < nr * b; e += BW_THREADS) sB[e / b][e % b] = B[(c0 + e / b) * ldb + e % b];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = tid + k * BW_THREADS;
      if (e < ne) {
        const int i = e / b, j = e % b;
        float s = 0.f;
        for (int rr = 0; rr < nr; ++rr) s = fmaf(sA[rr][i], sB[rr][j], s);
        acc[k] += (double)s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int e = tid + k * BW_THREADS;
    if (e < ne) part[(int64_t)g * ne + e] = acc[k];
  }
}

// out[e] = sum over the G partition partials (one block per entry e, a fixed reduction
// tree: deterministic); with a row stride ldo for the a x b result (ldo >= b).
constexpr int kSumThreads = 128;
__global__ void __launch_bounds__(kSumThreads)
k_cross_sum(const double* __restrict__ part, int G, int a, int b, double* __restrict__ out, int ldo, const int* skip) {
  if (block_skip(skip)) return;
  __shared__ double red[kSumThreads / 32];
  const int e = blockIdx.x, ne = a * b;
  double t = 0.0;
  for (int g = threadIdx.x; g < G; g += kSumThreads) t += part[(int64_t)g * ne + e];
  for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSumThreads / 32; ++w) s += red[w];
    out[(e / b) * ldo + e % b] = s;
  }
}

// C[i][c] = beta C[i][c] + alpha sum_l A[i][l] Bm[l][c] (Bm small, a x c, row stride ldbm;
// transposed: Bm[c][l]).  One thread per output entry; Bm staged in shared memory.
template <typename TB>
__global__ void __launch_bounds__(BW_THREADS)
k_tall_small(const float* __restrict__ A, int64_t lda, int a, const TB* __restrict__ Bm, int ldbm, int trans, int c,
             int64_t rows, float alpha, float beta, float* __restrict__ C, int64_t ldc, const int* skip) {
  if (block_skip(skip)) return;
  __shared__ float sB[kMaxRP][kMaxRP + 1];   // a, c <= 64
  for (int e = threadIdx.x; e < a * c; e += BW_THREADS) {
    const int l = e / c, cc = e % c;
    sB[l][cc] = (float)(trans ? Bm[cc * ldbm + l] : Bm[l * ldbm + cc]);
  }
  __syncthreads();
  const int64_t o = (int64_t)blockIdx.x * BW_THREADS + threadIdx.x;
  if (o >= rows * c) return;
  const int64_t i = o / c;
  const int cc = (int)(o % c);
  const float* ar = A + i * lda;
  float s = 0.f;
  for (int l = 0; l < a; ++l) s = fmaf(ar[l], sB[l][cc], s);
  float* cp = C + i * ldc + cc;
  *cp = (beta != 0.f ? beta * *cp : 0.f) + alpha * s;
}

// out[row][c] += v_e B[col][c] (or, transposed, out[col][c] += v_e B[row][c]) for the COO
// entries e (linear index row * n + col); float atomics.
__global__ void k_spmm(const int64_t* __restrict__ idx, const float* __restrict__ val, int64_t nnz, int64_t n,
                       const float* __restrict__ B, int64_t ldb, int c, int trans, float* __restrict__ out,
                       int64_t ldo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnz * c) return;
  const int64_t e = t / c;
  const int cc = (int)(t % c);
  const int64_t row = idx[e] / n, col = idx[e] % n;
  const float v = val[e];
  if (trans) atomicAdd(out + col * ldo + cc, v * B[row * ldb + cc]);
  else atomicAdd(out + row * ldo + cc, v * B[col * ldb + cc]);
}

// vals[e] = sum_c U[row][c] V[col][c] at the COO positions; with sub, also
// D[row][col] -= vals[e].
__global__ void k_eval_lr(const int64_t* __restrict__ idx, int64_t nnz, int64_t n, const float* __restrict__ U,
                          int64_t ldu, const float* __restrict__ V, int64_t ldv, int K, float* __restrict__ vals,
                          float* __restrict__ D, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int64_t row = idx[e] / n, col = idx[e] % n;
  const float* u = U + row * ldu;
  const float* v = V + col * ldv;
  float s = 0.f;
  for (int c = 0; c < K; ++c) s = fmaf(u[c], v[c], s);
  if (vals) vals[e] = s;
  if (D) D[row * ldd + col] -= s;
}

// Z[row][col] = vals[e] at the COO positions (Z holds a copy of X elsewhere).
__global__ void k_scatter_set(const int64_t* __restrict__ idx, const float* __restrict__ vals, int64_t nnz, int64_t n,
                              float* __restrict__ Z, int64_t ldz) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const int64_t row = idx[e] / n, col = idx[e] % n;
  Z[row * ldz + col] = vals[e];
}

// D (m x n) = beta D + U V^T, U m x K (ldu), V n x K (ldv), K <= 192: 128 x 128 output
// tiles, 256 threads each owning an 8 x 8 block (rows ty*4 + {0..3} and 64 + ty*4 + {0..3},
// the same for columns with tx), read from shared memory as float4s (four loads per 64
// fmas), K in chunks of 32 through shared memory; D read and written as float4s when its
// rows allow (ldd and the pointer 16-byte aligned), else element by element.
constexpr int OA_T = 128, OA_KC = 32, OA_LD = OA_T + 4;
__global__ void __launch_bounds__(BW_THREADS)
k_outer_acc(const float* __restrict__ U, int64_t ldu, const float* __restrict__ V, int64_t ldv, int K, int64_t m,
            int64_t n, float beta, float* __restrict__ D, int64_t ldd) {
  __shared__ __align__(16) float sU[OA_KC][OA_LD];
  __shared__ __align__(16) float sV[OA_KC][OA_LD];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t i0 = (int64_t)blockIdx.y * OA_T, j0 = (int64_t)blockIdx.x * OA_T;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < K; k0 += OA_KC) {
    __syncthreads();
    for (int e = tid; e < OA_KC * OA_T; e += BW_THREADS) {
      const int rr = e / OA_KC, kk = e % OA_KC;   // consecutive threads along k: rows of U / V are contiguous
      const int64_t gi = i0 + rr, gj = j0 + rr;
      sU[kk][rr] = (gi < m && k0 + kk < K) ? U[gi * ldu + k0 + kk] : 0.f;
      sV[kk][rr] = (gj < n && k0 + kk < K) ? V[gj * ldv + k0 + kk] : 0.f;
    }
    __syncthreads();
    const int kc = (K - k0 < OA_KC) ? K - k0 : OA_KC;
#pragma unroll 4
    for (int kk = 0; kk < kc; ++kk) {
      const float4 u0 = *reinterpret_cast<const float4*>(&sU[kk][ty * 4]);
      const float4 u1 = *reinterpret_cast<const float4*>(&sU[kk][64 + ty * 4]);
      const float4 v0 = *reinterpret_cast<const float4*>(&sV[kk][tx * 4]);
      const float4 v1 = *reinterpret_cast<const float4*>(&sV[kk][64 + tx * 4]);
      const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(u[a], v[b], acc[a][b]);
    }
  }
  const bool vec = ((ldd & 3) == 0) && ((reinterpret_cast<uintptr_t>(D) & 15) == 0);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int64_t gi = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
    if (gi >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t gj = j0 + h * 64 + tx * 4;
      float* d = D + gi * ldd + gj;
      const float* ac = &acc[a][4 * h];
      if (vec && gj + 3 < n) {
        float4 o = make_float4(ac[0], ac[1], ac[2], ac[3]);
        if (beta != 0.f) {
          const float4 p = *reinterpret_cast<const float4*>(d);
          o.x = fmaf(beta, p.x, o.x);
          o.y = fmaf(beta, p.y, o.y);
          o.z = fmaf(beta, p.z, o.z);
          o.w = fmaf(beta, p.w, o.w);
        }
        *reinterpret_cast<float4*>(d) = o;
      } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (gj + b < n) d[b] = (beta != 0.f ? beta * d[b] : 0.f) + ac[b];
      }
    }
  }
}

// y += alpha x
__global__ void k_axpy(const float* __restrict__ x, float* __restrict__ y, int64_t count, float alpha) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) y[i] = fmaf(alpha, x[i], y[i]);
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + BW_THREADS - 1) / BW_THREADS); }

}  // namespace

void launch_cross_gram(const float* A, int64_t lda, int a, const float* B, int64_t ldb, int b, int64_t rows,
                       double* part, int G, double* out, int ldo, cudaStream_t st, const int* skip) {
  if (a * b == 0) return;
  // about 128 rows per partition (short serial chains), at most the G the buffer holds
  int64_t gu = (rows + 127) / 128;
  if (gu > G) gu = G;
  if (gu < 1) gu = 1;
  k_cross_part<<<(unsigned)gu, BW_THREADS, 0, st>>>(A, lda, a, B, ldb, b, rows, part, skip);
  k_cross_sum<<<(unsigned)(a * b), kSumThreads, 0, st>>>(part, (int)gu, a, b, out, ldo, skip);
}

void launch_tall_small_f(const float* A, int64_t lda, int a, const float* Bm, int ldbm, int trans, int c, int64_t rows,
                         float alpha, float beta, float* C, int64_t ldc, cudaStream_t st, const int* skip) {
  if (rows * c == 0) return;
  k_tall_small<float><<<blocks_for(rows * c), BW_THREADS, 0, st>>>(A, lda, a, Bm, ldbm, trans, c, rows, alpha, beta,
                                                                   C, ldc, skip);
}

void launch_tall_small_d(const float* A, int64_t lda, int a, const double* Bm, int ldbm, int trans, int c,
                         int64_t rows, float alpha, float beta, float* C, int64_t ldc, cudaStream_t st,
                         const int* skip) {
  if (rows * c == 0) return;
  k_tall_small<double><<<blocks_for(rows * c), BW_THREADS, 0, st>>>(A, lda, a, Bm, ldbm, trans, c, rows, alpha, beta,
                                                                    C, ldc, skip);
}

void launch_spmm(const int64_t* idx, const float* val, int64_t nnz, int64_t n, const float* B, int64_t ldb, int c,
                 int trans, float* out, int64_t ldo, cudaStream_t st) {
  if (nnz * c == 0) return;
  k_spmm<<<blocks_for(nnz * c), BW_THREADS, 0, st>>>(idx, val, nnz, n, B, ldb, c, trans, out, ldo);
}

void launch_eval_lr(const int64_t* idx, int64_t nnz, int64_t n, const float* U, int64_t ldu, const float* V,
                    int64_t ldv, int K, float* vals, float* D, int64_t ldd, cudaStream_t st) {
  if (nnz == 0) return;
  k_eval_lr<<<blocks_for(nnz), BW_THREADS, 0, st>>>(idx, nnz, n, U, ldu, V, ldv, K, vals, D, ldd);
}

void launch_scatter_set(const int64_t* idx, const float* vals, int64_t nnz, int64_t n, float* Z, int64_t ldz,
                        cudaStream_t st) {
  if (nnz == 0) return;
  k_scatter_set<<<blocks_for(nnz), BW_THREADS, 0, st>>>(idx, vals, nnz, n, Z, ldz);
}

void launch_axpy(const float* x, float* y, int64_t count, float alpha, cudaStream_t st) {
  if (count > 0) k_axpy<<<blocks_for(count), BW_THREADS, 0, st>>>(x, y, count, alpha);
}

void launch_outer_acc(const float* U, int64_t ldu, const float* V, int64_t ldv, int K, int64_t m, int64_t n,
                      float beta, float* D, int64_t ldd, cudaStream_t st) {
  dim3 grid((unsigned)((n + OA_T - 1) / OA_T), (unsigned)((m + OA_T - 1) / OA_T));
  k_outer_acc<<<grid, BW_THREADS, 0, st>>>(U, ldu, V, ldv, K, m, n, beta, D, ldd);
}

}  // namespace godec
