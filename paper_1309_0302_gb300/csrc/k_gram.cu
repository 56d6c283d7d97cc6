// Gram partials of the 128-row tiles of a chain product's float32 output, for the rank
// test's exactly accumulated Gram of P = Z Q2 on the fast path: nothing on the critical path
// needs it, so it runs on the rank test's own stream (whose kernels have the GPU's few
// spare SMs to themselves while the chain goes on) instead of in the product's tile
// completion, where the double-float accumulation takes ~20 us.  Same partial layout as
// the product's own (tile t at t RP RP), summed by k_gram_sum.
#include "godec_internal.cuh"
#include "gram_tile.cuh"

namespace godec {

namespace {

constexpr int GT_ROWS = 128, GT_THREADS = 256, GT_LD = kMaxRP + 1;

// One block per tile; Y has row stride RP.
__global__ void __launch_bounds__(GT_THREADS)
k_gram_tiles(const float* __restrict__ Y, int64_t rows, int RP, int mode, void* __restrict__ part, const Ctl* ctl) {
  if (ctl && ctl->abort) return;
  __shared__ float Ps[GT_ROWS * GT_LD];
  const int tid = threadIdx.x;
  const int64_t t = blockIdx.x, o0 = t * GT_ROWS;
  const int nrow = (int)(rows - o0 < GT_ROWS ? rows - o0 : GT_ROWS);
  for (int e = tid; e < GT_ROWS * RP; e += GT_THREADS) {
    const int i = e / RP, l = e % RP;
    Ps[i * GT_LD + l] = i < nrow ? __ldcg(Y + (o0 + i) * RP + l) : 0.f;
  }
  __syncthreads();
  const size_t esz = mode == 2 ? sizeof(double) : sizeof(float);
  gram_tile(Ps, GT_LD, RP, mode, static_cast<char*>(part) + (size_t)t * RP * RP * esz, tid, GT_THREADS);
}

}  // namespace

void launch_gram_tiles(const float* Y, int64_t rows, int RP, int mode, void* part, const Ctl* ctl, cudaStream_t st) {
  const int64_t tiles = (rows + GT_ROWS - 1) / GT_ROWS;
  k_gram_tiles<<<(unsigned)tiles, GT_THREADS, 0, st>>>(Y, rows, RP, mode, part, ctl);
}

}  // namespace godec
