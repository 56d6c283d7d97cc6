// Small helpers: zero fill, padded copies of tall factors, ||X||_F^2 and a
// stable LSD radix sort of the COO of S by linear index (export order).
#include <algorithm>

#include "godec_internal.cuh"
#include "tc_util.cuh"

namespace godec {

namespace {

__global__ void k_fill_zero(uint4* p, size_t n16) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    p[i] = make_uint4(0, 0, 0, 0);
}

// 32 x 32 tiles through shared memory (padded against bank conflicts)
__global__ void k_transpose(const float* __restrict__ src, int64_t m, int64_t n, int64_t lds,
                            float* __restrict__ dst, int64_t ldd, const float* __restrict__ scale) {
  __shared__ float t[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const float sc = scale ? scale[0] : 1.f;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t i = i0 + k, j = j0 + threadIdx.x;
    t[k][threadIdx.x] = (i < m && j < n) ? src[i * lds + j] * sc : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int64_t j = j0 + k, i = i0 + threadIdx.x;
    if (j < n && i < m) dst[j * ldd + i] = t[threadIdx.x][k];
  }
}

__global__ void k_pad_copy(const float* src, int64_t rows, int cols, int64_t lds, float* dst, int RP) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * RP;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / RP;
    int c = (int)(e % RP);
    dst[e] = (c < cols) ? src[i * lds + c] : 0.f;
  }
}

__global__ void k_unpad_copy(const float* src, int64_t rows, int RP, float* dst, int cols) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / cols;
    int c = (int)(e % cols);
    dst[e] = src[i * RP + c];
  }
}

__global__ void k_sumsq(const float* X, int64_t m, int64_t n, int64_t ldx, double* out) {
  double acc = 0.0;
  const int64_t total = m * n;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 16; base < total;
       base += (int64_t)gridDim.x * blockDim.x * 16) {
    float f = 0.f;
    for (int64_t e = base; e < min(total, base + 16); ++e) {
      int64_t i = e / n, j = e % n;
      float v = X[i * ldx + j];
      f = fmaf(v, v, f);
    }
    acc += (double)f;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// ---- LSD radix sort, 4-bit digits, items owned contiguously by threads (stable) ------
constexpr int SORT_THREADS = 256, SORT_ITEMS = 16, SORT_TILE = SORT_THREADS * SORT_ITEMS;

__global__ void k_scale_copy(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                             const float* scale) {
  const float sc = scale[0];
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) dst[r * ldd + c] = src[r * lds + c] * sc;
}

__global__ void k_scale_update(float* zscale, const float* f) {
  zscale[0] *= f[0];
  zscale[1] *= f[1];
}

// max |Z| over the matrix (non-negative floats order like their bit patterns).
__global__ void k_maxabs(const float* Z, int64_t rows, int64_t cols, int64_t ld, unsigned* out) {
  float m = 0.f;
  for (int64_t r = blockIdx.x; r < rows; r += gridDim.x)
    for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) m = fmaxf(m, fabsf(Z[r * ld + c]));
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

__global__ void k_make_zscale(const unsigned* mx, float* zscale) {
  const float m = __uint_as_float(*mx);
  int e = 0;
  if (m > 0.f && isfinite(m)) {
    int ex;
    frexpf(m, &ex);   // m in [2^(ex-1), 2^ex)
    e = 13 - ex;
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
  }
  zscale[0] = ldexpf(1.f, e);
  zscale[1] = ldexpf(1.f, -e);
}

__global__ void k_sort_hist(const long long* keys, long long n, int shift, unsigned* cnt, int nblk) {
  __shared__ unsigned h[16];
  if (threadIdx.x < 16) h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * SORT_TILE;
  for (int j = threadIdx.x; j < SORT_TILE; j += SORT_THREADS) {
    long long e = base + j;
    if (e < n) atomicAdd(&h[(keys[e] >> shift) & 15], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 16) cnt[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_sort_scan(unsigned* cnt, int total) {
  // single block exclusive scan of `total` counts (digit-major), 1024 threads
  __shared__ unsigned carry;
  __shared__ unsigned ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < total; base += 1024) {
    int i = base + threadIdx.x;
    unsigned v = i < total ? cnt[i] : 0u;
    unsigned x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned s = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    unsigned excl = carry + (w ? ws[w - 1] : 0u) + x - v;
    if (i < total) cnt[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void k_sort_scatter(const long long* kin, const float* vin, long long* kout, float* vout,
                               long long n, int shift, const unsigned* off, int nblk) {
  __shared__ unsigned tab[16][SORT_THREADS + 1];
  const int t = threadIdx.x;
  const long long base = (long long)blockIdx.x * SORT_TILE + (long long)t * SORT_ITEMS;
  unsigned c[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) c[d] = 0;
  long long kk[SORT_ITEMS];
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j) {
    long long e = base + j;
    kk[j] = e < n ? kin[e] : -1;
    if (e < n) c[(kk[j] >> shift) & 15]++;
  }
#pragma unroll
  for (int d = 0; d < 16; ++d) tab[d][t] = c[d];
  __syncthreads();
  // exclusive scan of each digit row across the 256 threads: warp w scans rows 2w, 2w+1
  const int lane = t & 31, w = t >> 5;
  for (int d = 2 * w; d < 2 * w + 2; ++d) {
    unsigned run = 0;
    unsigned vals[8];
    for (int j = 0; j < 8; ++j) { vals[j] = tab[d][lane * 8 + j]; run += vals[j]; }
    unsigned x = run;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    unsigned e = x - run;
    for (int j = 0; j < 8; ++j) { tab[d][lane * 8 + j] = e; e += vals[j]; }
  }
  __syncthreads();
  unsigned pos[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) pos[d] = off[d * nblk + blockIdx.x] + tab[d][t];
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j) {
    long long e = base + j;
    if (e < n) {
      int d = (int)((kk[j] >> shift) & 15);
      unsigned p = pos[d]++;
      kout[p] = kk[j];
      vout[p] = vin[e];
    }
  }
}

// Self-test of the timeout path: thread 0 waits, with the pipelines' bounded polling
// helper, on a fresh mbarrier that nothing arrives on, and gives up after `polls` polls
// (each at most tc::kPollNs) as a pipeline wait does: it flags the context (timeout,
// abort) and returns.  Nothing is left in flight.
__global__ void k_wait_check(Ctl* ctl, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  tc::fence_barrier_init();
  if (!tc::mbar_wait(&bar, 0u, polls)) {
    ctl->timeout = 1;
    ctl->abort = 1;
  }
}

}  // namespace

void launch_wait_check(Ctl* ctl, uint32_t polls, cudaStream_t st) { k_wait_check<<<1, 32, 0, st>>>(ctl, polls); }

void launch_fill_zero(void* p, size_t bytes, cudaStream_t st) {
  // bytes must be a multiple of 16 and p 16-byte aligned
  size_t n16 = bytes / 16;
  if (!n16) return;
  unsigned grid = (unsigned)std::min<size_t>((n16 + 255) / 256, 4096);
  k_fill_zero<<<grid, 256, 0, st>>>(reinterpret_cast<uint4*>(p), n16);
}

void launch_transpose(const float* src, int64_t m, int64_t n, int64_t lds, float* dst, int64_t ldd,
                      cudaStream_t st, const float* scale) {
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
  k_transpose<<<grid, dim3(32, 8), 0, st>>>(src, m, n, lds, dst, ldd, scale);
}

void launch_pad_copy(const float* src, int64_t rows, int cols, int64_t lds, float* dst, int RP,
                     cudaStream_t st) {
  int64_t tot = rows * RP;
  unsigned grid = (unsigned)std::min<int64_t>((tot + 255) / 256, 4096);
  if (grid) k_pad_copy<<<grid, 256, 0, st>>>(src, rows, cols, lds, dst, RP);
}

void launch_unpad_copy(const float* src, int64_t rows, int RP, float* dst, int cols, cudaStream_t st) {
  int64_t tot = rows * cols;
  unsigned grid = (unsigned)std::min<int64_t>((tot + 255) / 256, 4096);
  if (grid) k_unpad_copy<<<grid, 256, 0, st>>>(src, rows, RP, dst, cols);
}

void launch_sumsq(const float* X, int64_t m, int64_t n, int64_t ldx, double* out, int nsm,
                  cudaStream_t st) {
  k_sumsq<<<(unsigned)(4 * nsm), 256, 0, st>>>(X, m, n, ldx, out);
}

size_t sort_coo_scratch(long long nnz) {
  long long nblk = (nnz + SORT_TILE - 1) / SORT_TILE;
  return (size_t)nnz * (sizeof(long long) + sizeof(float)) + (size_t)(16 * nblk + 16) * sizeof(unsigned) + 256;
}

void launch_zscale(const float* Z, int64_t rows, int64_t cols, int64_t ld, unsigned* zmax, float* zscale, int nsm,
                   cudaStream_t st) {
  cudaMemsetAsync(zmax, 0, sizeof(unsigned), st);
  int64_t grid = 4LL * nsm;
  if (grid > rows) grid = rows;
  k_maxabs<<<(unsigned)grid, 256, 0, st>>>(Z, rows, cols, ld, zmax);
  k_make_zscale<<<1, 1, 0, st>>>(zmax, zscale);
}

void launch_scale_copy(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                       const float* scale, int nsm, cudaStream_t st) {
  int64_t grid = 4LL * nsm;
  if (grid > rows) grid = rows;
  k_scale_copy<<<(unsigned)grid, 256, 0, st>>>(src, rows, cols, lds, dst, ldd, scale);
}

void launch_scale_update(float* zscale, const float* f, cudaStream_t st) { k_scale_update<<<1, 1, 0, st>>>(zscale, f); }

void launch_sort_coo(long long* idx, float* val, long long nnz, void* scratch, size_t scratch_bytes,
                     int idx_bits, cudaStream_t st) {
  if (nnz <= 1) return;
  const int nblk = (int)((nnz + SORT_TILE - 1) / SORT_TILE);
  char* p = reinterpret_cast<char*>(scratch);
  long long* k2 = reinterpret_cast<long long*>(p);
  float* v2 = reinterpret_cast<float*>(p + (size_t)nnz * sizeof(long long));
  size_t offb = (size_t)nnz * (sizeof(long long) + sizeof(float));
  offb = (offb + 255) & ~size_t(255);
  unsigned* cnt = reinterpret_cast<unsigned*>(p + offb);
  (void)scratch_bytes;
  long long* ka = idx;
  float* va = val;
  long long* kb = k2;
  float* vb = v2;
  int passes = (idx_bits + 3) / 4;
  if (passes & 1) ++passes;                  // even count: result lands back in idx/val
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = 4 * ps;
    k_sort_hist<<<nblk, SORT_THREADS, 0, st>>>(ka, nnz, shift, cnt, nblk);
    k_sort_scan<<<1, 1024, 0, st>>>(cnt, 16 * nblk);
    k_sort_scatter<<<nblk, SORT_THREADS, 0, st>>>(ka, va, kb, vb, nnz, shift, cnt, nblk);
    long long* tk = ka; ka = kb; kb = tk;
    float* tv = va; va = vb; vb = tv;
  }
}

}  // namespace godec
