// First projection of the power chain from a cached X A1.
//
// The chain's first product is Y1 = (X - S) A1 (Algorithm 1's L-step), and the test matrix A1
// stays fixed across iterations (only a rank drop zeroes some of its columns).  With S
// held on its support of k entries, (X - S) A1 = X A1 - S A1: X A1 is formed once, by the
// tensor-core product over X, and each iteration subtracts S A1, k r multiply-adds,
// instead of streaming the m x n matrix Z.
//
// S is read on its support bitmap (bit i n + j for entry (i, j)) as X - Z / s_Z: Z holds
// (X - S) s_Z on the support, so this is the value the product over Z would have used.
// Each row is handled by 16 lanes (two rows per warp, four columns of A1 per lane): the
// row's bitmap words are staged in shared memory in one round trip and expanded into a
// list of columns in increasing order, the entries' values gathered together, and the A1
// rows subtracted in column order, so the result does not depend on the schedule.  The
// work is a chain of memory round trips per row, so the blocks are small and every row of
// a 10^4-row matrix is resident at once.
#include "godec_internal.cuh"

namespace godec {
namespace {

constexpr int SP_WARPS = 2;            // two rows per warp
constexpr int SP_WCAP = 320;           // bitmap words of a row staged at a time (10240 columns)
constexpr int SP_CAP = 192;            // listed entries of a row applied at a time
constexpr int SP_AHEAD = 8;            // A1 rows in flight per row

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

__global__ void __launch_bounds__(SP_WARPS * 32, 18)   // 36 warps, 72 rows per SM
k_sproj(const float* __restrict__ XA1, const float* __restrict__ A1, int RP, const float* __restrict__ X, int64_t ldx,
        const float* __restrict__ Z, int64_t ldz, int64_t m, int64_t n, const unsigned* __restrict__ sbits,
        long long words, Ctl* __restrict__ ctl, float* __restrict__ P) {
  __shared__ unsigned s_w[SP_WARPS * 2][SP_WCAP];
  __shared__ int s_j[SP_WARPS * 2][SP_CAP];
  __shared__ float s_v[SP_WARPS * 2][SP_CAP];
  if (ctl->abort) return;
  if (ctl->range_err) {   // the last S-step left Z out of the product's range: as the product would
    if (threadIdx.x == 0) ctl->abort = 1;
    return;
  }
  // No early return below: both halves of a warp take part in every shuffle, and every
  // branch around one is taken by the whole warp.
  const unsigned full = 0xffffffffu;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, hl = lane & 15;
  const int slot = warp * 2 + (lane >> 4);
  const int64_t i = ((int64_t)blockIdx.x * SP_WARPS + warp) * 2 + (lane >> 4);
  const bool live = i < m;
  const bool colok = live && 4 * hl < RP;   // RP is a multiple of 8: float4 columns
  const unsigned* B = sbits + (size_t)ctl->cur * (size_t)words;
  const float zi = ctl->zscale[1];
  float4 acc = colok ? *reinterpret_cast<const float4*>(XA1 + i * RP + 4 * hl) : make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t b0 = i * n, b1 = b0 + n;   // the row's bits [b0, b1)
  const int64_t w0 = b0 >> 5;
  const int64_t nw = live ? ((b1 - 1) >> 5) - w0 + 1 : 0;
  const int64_t nwmax = n / 32 + 2;         // bound on nw for every row (uniform)
  const float* Xr = X + (live ? i : 0) * ldx;
  const float* Zr = Z + (live ? i : 0) * ldz;
  int* lj = s_j[slot];
  float* lv = s_v[slot];
  // Applies the nl listed entries of this row (called by the whole warp).
  auto apply = [&](int nl) {
    __syncwarp();
    const int cm = max(nl, __shfl_xor_sync(full, nl, 16));
    for (int u0 = 0; u0 < cm; u0 += 16 * 8) {   // S on the entries, 8 gathers in flight per lane
      float xv[8], zv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = u0 + 16 * u + hl;
        xv[u] = zv[u] = 0.f;
        if (e < nl) {
          const int j = lj[e];
          xv[u] = Xr[j];
          zv[u] = Zr[j];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = u0 + 16 * u + hl;
        if (e < nl) lv[e] = xv[u] - zv[u] * zi;
      }
    }
    __syncwarp();
    for (int t0 = 0; t0 < cm; t0 += SP_AHEAD) {
      float4 a[SP_AHEAD];
      float sv[SP_AHEAD];
#pragma unroll
      for (int u = 0; u < SP_AHEAD; ++u) {
        const bool ok = t0 + u < nl;
        const int j = ok ? lj[t0 + u] : 0;
        sv[u] = ok ? lv[t0 + u] : 0.f;
        a[u] = (ok && colok) ? __ldg(reinterpret_cast<const float4*>(A1 + (int64_t)j * RP + 4 * hl))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < SP_AHEAD; ++u)
        if (t0 + u < nl) {
          acc.x = fmaf(-sv[u], a[u].x, acc.x);
          acc.y = fmaf(-sv[u], a[u].y, acc.y);
          acc.z = fmaf(-sv[u], a[u].z, acc.z);
          acc.w = fmaf(-sv[u], a[u].w, acc.w);
        }
    }
    __syncwarp();
  };
  int nl = 0;   // entries listed and not yet applied
  for (int64_t c0 = 0; c0 < nwmax; c0 += SP_WCAP) {
    // the chunk's words into shared memory in one round trip
    const int nwc = (int)max((int64_t)0, min(nw - c0, (int64_t)SP_WCAP));
    for (int r = hl; r < nwc; r += 16) cp_async4(&s_w[slot][r], B + w0 + c0 + r);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    const int nit = (int)((min(nwmax - c0, (int64_t)SP_WCAP) + 15) / 16);
    for (int t = 0; t < nit; ++t) {
      // 16 consecutive words per step, one per lane; their set bits in order
      const int r = 16 * t + hl;
      unsigned x = 0u;
      if (r < nwc) {
        x = s_w[slot][r];
        const int64_t rr = c0 + r;
        if (rr == 0) x &= ~0u << (int)(b0 & 31);
        if (rr == nw - 1) {
          const int hb = (int)((b1 - 1) & 31);
          x &= hb == 31 ? ~0u : ((2u << hb) - 1u);
        }
      }
      const int c = __popc(x);
      int inc = c;
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const int y = __shfl_up_sync(full, inc, o, 16);
        if (hl >= o) inc += y;
      }
      const int tot = __shfl_sync(full, inc, 15, 16);   // <= 512
      const int64_t colb = (w0 + c0 + r) * 32 - b0;   // column of bit 0 of this lane's word
      if (__any_sync(full, nl + tot > SP_CAP)) {
        apply(nl);
        nl = 0;
      }
      // list the step's entries with positions [lo, lo + SP_CAP) (more rounds if it has more)
      for (int lo = 0; lo < 512; lo += SP_CAP) {
        if (!__any_sync(full, tot > lo)) break;
        if (lo) {
          apply(nl);
          nl = 0;
        }
        unsigned y = x;
        int pos = inc - c;
        while (y) {
          const int b = __ffs(y) - 1;
          y &= y - 1u;
          const int q = pos - lo;
          if (q >= 0 && q < SP_CAP) lj[nl + q] = (int)(colb + b);
          ++pos;
        }
        nl += max(0, min(tot - lo, SP_CAP));
      }
    }
    __syncwarp();   // the words are read before the next chunk overwrites them
  }
  apply(nl);
  if (colok) *reinterpret_cast<float4*>(P + i * RP + 4 * hl) = acc;
}

}  // namespace

void launch_sproj(const float* XA1, const float* A1, int RP, const float* X, int64_t ldx, const float* Z, int64_t ldz,
                  int64_t m, int64_t n, const unsigned* sbits, long long words, Ctl* ctl, float* P,
                  cudaStream_t st) {
  const unsigned grid = (unsigned)((m + 2 * SP_WARPS - 1) / (2 * SP_WARPS));
  k_sproj<<<grid, SP_WARPS * 32, 0, st>>>(XA1, A1, RP, X, ldx, Z, ldz, m, n, sbits, words, ctl, P);
}

}  // namespace godec
