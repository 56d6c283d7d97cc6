// Dense form of the low-rank part: L = U diag(sigma) V^T (eq. mlr_app, L = Q1 M^{1/(2q+1)}
// Q2^T, whose factors the L-step keeps).  The iteration never forms L; this kernel is for
// callers that need it as a matrix (the differentiated form's output, a dense loss).
//
// One block of 256 threads writes a 64-row x 128-column tile.  The tile's rows of
// U diag(sigma) and columns of V^T are staged in shared memory; each thread accumulates a
// 4 x 8 block (rows ty + 16a, columns 4 tx + {0..3} and 64 + 4 tx + {0..3}) in float32 and
// writes it with 16-byte stores where the row stride allows (a warp then covers two rows
// of 256 contiguous bytes).  Bound: the 4 m n bytes written (plus 2 m n r flops).
#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int DT_ROWS = 64, DT_COLS = 128, DT_THREADS = 256;

__global__ void __launch_bounds__(DT_THREADS)
k_lowrank_dense(const float* __restrict__ U, int64_t ldu, const float* __restrict__ sigma,
                const float* __restrict__ V, int64_t ldv, int64_t m, int64_t n, int r, float* __restrict__ L,
                int64_t ldl, int vec4) {
  __shared__ float Ut[kMaxRP][DT_ROWS];                 // (U diag(sigma))^T, tile rows
  __shared__ __align__(16) float Vt[kMaxRP][DT_COLS];   // V^T, tile columns (48 KB in all)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t ncolt = (n + DT_COLS - 1) / DT_COLS;
  const int64_t i0 = (int64_t)(blockIdx.x / ncolt) * DT_ROWS, j0 = (int64_t)(blockIdx.x % ncolt) * DT_COLS;
  for (int e = tid; e < DT_ROWS * r; e += DT_THREADS) {
    const int i = e / r, l = e % r;
    Ut[l][i] = (i0 + i < m) ? U[(i0 + i) * ldu + l] * sigma[l] : 0.f;
  }
  for (int e = tid; e < DT_COLS * r; e += DT_THREADS) {
    const int j = e / r, l = e % r;
    Vt[l][j] = (j0 + j < n) ? V[(j0 + j) * ldv + l] : 0.f;
  }
  __syncthreads();
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int l = 0; l < r; ++l) {
    const float4 v0 = *reinterpret_cast<const float4*>(&Vt[l][4 * tx]);
    const float4 v1 = *reinterpret_cast<const float4*>(&Vt[l][64 + 4 * tx]);
    const float bv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float u = Ut[l][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(u, bv[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + ty + 16 * a;
    if (i >= m) continue;
    float* row = L + i * ldl;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t j = j0 + 64 * h + 4 * tx;
      if (vec4 && j + 3 < n) {
        *reinterpret_cast<float4*>(row + j) =
            make_float4(acc[a][4 * h], acc[a][4 * h + 1], acc[a][4 * h + 2], acc[a][4 * h + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (j + c < n) row[j + c] = acc[a][4 * h + c];
      }
    }
  }
}

}  // namespace

void launch_lowrank_dense(const float* U, int64_t ldu, const float* sigma, const float* V, int64_t ldv, int64_t m,
                          int64_t n, int r, float* L, int64_t ldl, cudaStream_t st) {
  if (r <= 0) {
    cudaMemset2DAsync(L, (size_t)ldl * sizeof(float), 0, (size_t)n * sizeof(float), (size_t)m, st);
    return;
  }
  const int vec4 = (ldl % 4 == 0) && (reinterpret_cast<uintptr_t>(L) % 16 == 0);
  // one block per tile, row-major over the tiles (m n < 2^32 keeps this below 2^31 blocks)
  const int64_t tiles = ((n + DT_COLS - 1) / DT_COLS) * ((m + DT_ROWS - 1) / DT_ROWS);
  k_lowrank_dense<<<(unsigned)tiles, DT_THREADS, 0, st>>>(U, ldu, sigma, V, ldv, m, n, r, L, ldl, vec4);
}

}  // namespace godec
