// S-step of Algorithm 1 (eq. raw_lss): S_t = P_Omega(X - L_t) with Omega
// the nonzero subset of the k largest |X - L_t|, ties by ascending linear index.
//
// One pass over X rebuilds R = X - U diag(sigma) V^T tile by tile.  Magnitudes
// are compared through their float bit patterns (monotone for |R| >= 0).  In
// candidate mode the pass keeps every entry whose key reaches a threshold
// guessed from the previous iteration; in full mode it builds a 4096-bin
// histogram of the top 12 key bits instead.  A short radix select over the
// candidates (3 key digits, then up to 4 index digits for ties) yields the
// exact k-th key and the tie cut, and the emit step writes S as COO.
#include <cuda_bf16.h>

#include <cuda_fp16.h>

#include "godec_internal.cuh"

namespace godec {

namespace {

constexpr int RT_M = 128, RT_N = 64, RES_THREADS = 128;
constexpr int RES_US_STRIDE = RT_M + 4, RES_VS_STRIDE = RT_N + 4;
constexpr size_t kResSmem = (size_t)kMaxRP * (RES_US_STRIDE + RES_VS_STRIDE) * sizeof(float) +
                            kHistBins * sizeof(unsigned);

__device__ __forceinline__ unsigned key_of(float v) { return __float_as_uint(v) & 0x7fffffffu; }

// Block-wide exclusive scan of one unsigned per thread (any blockDim multiple of 32).
__device__ unsigned block_excl_scan(unsigned v, unsigned* total) {
  __shared__ unsigned wsum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) wsum[lane] = w;
  }
  __syncthreads();
  unsigned before = warp ? wsum[warp - 1] : 0u;
  *total = wsum[nw - 1];
  return before + x - v;
}

__device__ double block_sum_double(double v) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) ws[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += ws[w];
  return t;   // valid in thread 0
}

// --------------------------------------------------------------------------------------
// Residual pass
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(RES_THREADS)
k_residual(ResidualArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort) return;
  const int mode = ctl->plan[a.pass];
  if (mode == PASS_NONE) return;
  const unsigned guess = ctl->guess[a.pass];
  extern __shared__ __align__(16) float res_smem[];
  float* Us = res_smem;                                  // [RP][RES_US_STRIDE]
  float* Vs = Us + kMaxRP * RES_US_STRIDE;               // [RP][RES_VS_STRIDE]
  unsigned* hist = reinterpret_cast<unsigned*>(Vs + kMaxRP * RES_VS_STRIDE);

  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;
  const int r = a.r, RP = a.RP;
  const int64_t m = a.m, n = a.n, ldx = a.ldx;
  const int64_t tiles_n = (n + RT_N - 1) / RT_N;
  const int64_t ntiles = ((m + RT_M - 1) / RT_M) * tiles_n;

  if (mode == PASS_FULL)
    for (int b = tid; b < kHistBins; b += RES_THREADS) hist[b] = 0u;

  double dsum = 0.0;
  int bad = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = (tile / tiles_n) * RT_M;
    const int64_t j0 = (tile % tiles_n) * RT_N;
    __syncthreads();
    for (int e = tid; e < RT_M * r; e += RES_THREADS) {
      int ii = e / r, l = e % r;
      int64_t i = i0 + ii;
      Us[l * RES_US_STRIDE + ii] = (i < m) ? a.U[i * RP + l] * a.sigma[l] : 0.f;
    }
    for (int e = tid; e < RT_N * r; e += RES_THREADS) {
      int jj = e / r, l = e % r;
      int64_t j = j0 + jj;
      Vs[l * RES_VS_STRIDE + jj] = (j < n) ? a.V[j * RP + l] : 0.f;
    }
    __syncthreads();
    float acc[8][8];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
    for (int l = 0; l < r; ++l) {
      float4 u0 = *reinterpret_cast<const float4*>(&Us[l * RES_US_STRIDE + ty * 8]);
      float4 u1 = *reinterpret_cast<const float4*>(&Us[l * RES_US_STRIDE + ty * 8 + 4]);
      float4 v0 = *reinterpret_cast<const float4*>(&Vs[l * RES_VS_STRIDE + tx * 8]);
      float4 v1 = *reinterpret_cast<const float4*>(&Vs[l * RES_VS_STRIDE + tx * 8 + 4]);
      float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(uv[p], vv[q], acc[p][q]);
    }
    // residual R = X - L on the 8 x 8 register tile
    const int64_t jb = j0 + tx * 8;
    unsigned ncand = 0;
    float fsum = 0.f;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int64_t i = i0 + ty * 8 + p;
      float xv[8];
      if (i < m && jb + 8 <= n) {
        const float4* xp = reinterpret_cast<const float4*>(a.X + i * ldx + jb);
        float4 x0 = xp[0], x1 = xp[1];
        xv[0] = x0.x; xv[1] = x0.y; xv[2] = x0.z; xv[3] = x0.w;
        xv[4] = x1.x; xv[5] = x1.y; xv[6] = x1.z; xv[7] = x1.w;
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) xv[q] = (i < m && jb + q < n) ? a.X[i * ldx + jb + q] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool in = (i < m) && (jb + q < n);
        float res = in ? xv[q] - acc[p][q] : 0.f;
        acc[p][q] = res;
        unsigned key = key_of(res);
        if (key >= 0x7f800000u) bad = 1;
        if (mode == PASS_FULL) {
          fsum = fmaf(res, res, fsum);
          if (key) atomicAdd(&hist[key >> kD1Shift], 1u);
        } else if (key != 0u && key >= guess) {
          ++ncand;
        } else {
          fsum = fmaf(res, res, fsum);
        }
      }
    }
    dsum += (double)fsum;
    if (mode == PASS_CAND) {
      unsigned total;
      unsigned off = block_excl_scan(ncand, &total);
      __shared__ unsigned long long s_base;
      if (tid == 0) s_base = total ? atomicAdd(&ctl->cand_count, (unsigned long long)total) : 0ull;
      __syncthreads();
      if (ncand) {
        unsigned long long pos = s_base + off;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const int64_t i = i0 + ty * 8 + p;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float res = acc[p][q];
            unsigned key = key_of(res);
            if (key != 0u && key >= guess) {
              if (pos < a.cand_cap) {
                a.cand_key[pos] = key;
                a.cand_idx[pos] = (long long)(i * n + jb + q);
                a.cand_val[pos] = res;
              }
              ++pos;
            }
          }
        }
      }
    }
  }
  if (bad) ctl->nonfinite = 1;
  double t = block_sum_double(dsum);
  if (tid == 0) atomicAdd(mode == PASS_FULL ? &ctl->sumsq_full : &ctl->sumsq_noncand, t);
  if (mode == PASS_FULL) {
    __syncthreads();
    for (int b = tid; b < kHistBins; b += RES_THREADS)
      if (hist[b]) atomicAdd(&ctl->hist[b], hist[b]);
  }
}

// --------------------------------------------------------------------------------------
// Pass control (one block of 1024 threads): decide what the next residual pass does.
// --------------------------------------------------------------------------------------
constexpr int CTL_THREADS = 1024;

// Find the bin holding the `need`-th largest (from_top) or smallest (!from_top) element of a
// histogram of `nb` bins (nb <= 4096).  Returns the bin; *above = elements strictly before it
// in that order, *in_bin = its count.  All threads get the result.
__device__ int block_find_bin(const unsigned* h, int nb, unsigned long long need, bool from_top,
                              unsigned long long* before, unsigned* in_bin,
                              unsigned long long* total_out) {
  __shared__ int s_bin;
  __shared__ unsigned long long s_before;
  __shared__ unsigned s_in;
  __shared__ unsigned long long s_total;
  const int per = (nb + CTL_THREADS - 1) / CTL_THREADS;   // bins per thread (<= 4)
  const int t = threadIdx.x;
  // thread t owns ordered positions [t*per, t*per+per); position o maps to bin
  // from_top ? nb-1-o : o
  unsigned loc = 0;
  for (int o = t * per; o < min(nb, t * per + per); ++o) loc += h[from_top ? nb - 1 - o : o];
  unsigned tot32;
  unsigned excl = block_excl_scan(loc, &tot32);
  if (t == 0) { s_bin = -1; s_total = tot32; }
  __syncthreads();
  unsigned long long run = excl;
  for (int o = t * per; o < min(nb, t * per + per); ++o) {
    int b = from_top ? nb - 1 - o : o;
    unsigned c = h[b];
    if (run < need && run + c >= need) {
      s_bin = b;
      s_before = run;
      s_in = c;
    }
    run += c;
  }
  __syncthreads();
  *before = s_before;
  *in_bin = s_in;
  *total_out = s_total;
  return s_bin;
}

__global__ void __launch_bounds__(CTL_THREADS)
k_after_pass(Ctl* ctl, int pass, long long k, unsigned long long cap) {
  if (ctl->abort) return;
  const int mode = ctl->plan[pass];
  if (mode == PASS_NONE || ctl->ready) return;
  const int t = threadIdx.x;
  if (mode == PASS_FULL) {
    unsigned long long before, total;
    unsigned in_bin;
    // total count first (need = 1 finds the top non-empty bin; we only want the total)
    block_find_bin(ctl->hist, kHistBins, 1ull, true, &before, &in_bin, &total);
    long long keff = (long long)((unsigned long long)k < total ? (unsigned long long)k : total);
    int bin = -1;
    if (keff > 0) bin = block_find_bin(ctl->hist, kHistBins, (unsigned long long)keff, true,
                                       &before, &in_bin, &total);
    __syncthreads();
    for (int b = t; b < kHistBins; b += CTL_THREADS) ctl->hist[b] = 0u;
    if (t == 0) {
      ctl->k_eff = keff;
      if (ctl->nonfinite) {
        ctl->abort = 1;
      } else if (keff == 0) {
        ctl->ready = 1;
        ctl->need = 0;
        ctl->cand_count = 0;
        ctl->sumsq_noncand = ctl->sumsq_full;
      } else {
        unsigned long long ge = before + in_bin;   // keys in bins >= bin
        if (ge > cap) {
          ctl->need_bigger_cand = 1;
          ctl->abort = 1;
        } else if (pass < 2) {
          ctl->plan[pass + 1] = PASS_CAND;
          unsigned g = (unsigned)bin << kD1Shift;
          ctl->guess[pass + 1] = g ? g : 1u;
          ctl->cand_count = 0;
          ctl->sumsq_noncand = 0.0;
        } else {
          ctl->abort = 1;                          // cannot happen: FULL is never last
        }
      }
    }
  } else if (t == 0) {   // PASS_CAND
    unsigned long long cc = ctl->cand_count;
    if (ctl->nonfinite) {
      ctl->abort = 1;
    } else if (cc <= cap && (long long)cc >= ctl->k_eff) {
      ctl->ready = 1;
      ctl->need = ctl->k_eff;
    } else if (pass < 2) {
      ctl->plan[pass + 1] = PASS_FULL;
      ctl->cand_count = 0;
      ctl->sumsq_full = 0.0;
    } else {
      ctl->need_bigger_cand = 1;
      ctl->abort = 1;
    }
  }
  if (t == 0) ctl->passes_run = pass + 1;
}

// --------------------------------------------------------------------------------------
// Radix select rounds over the candidates.  Round 0..2: key digits (bits 30..19, 18..7,
// 6..0), largest first.  Rounds 3..6: 12-bit digits of the linear index of the ties,
// smallest first.  The last block to finish scans the histogram.
// --------------------------------------------------------------------------------------
constexpr int SEL_THREADS = 512;

__device__ __forceinline__ void round_digit(int round, int* shift, int* bits) {
  switch (round) {
    case 0: *shift = 19; *bits = 12; break;
    case 1: *shift = 7; *bits = 12; break;
    case 2: *shift = 0; *bits = 7; break;
    default: *shift = 12 * (6 - round); *bits = 12; break;   // 36, 24, 12, 0
  }
}

__global__ void __launch_bounds__(SEL_THREADS)
k_select_round(SelectArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort || !ctl->ready || ctl->need <= 0) return;
  const int round = a.round;
  if (round < 3 && ctl->key_done) return;
  if (round >= 3) {
    if (!ctl->key_done || ctl->idx_done) return;
    int sh, bt;
    round_digit(round, &sh, &bt);
    if (sh >= a.idx_bits && round < 6) return;     // digit is zero for every index
  }
  __shared__ unsigned h[kHistBins];
  const int tid = threadIdx.x;
  for (int b = tid; b < kHistBins; b += SEL_THREADS) h[b] = 0u;
  __syncthreads();
  int shift, bits;
  round_digit(round, &shift, &bits);
  const unsigned long long ncand = min(ctl->cand_count, a.cand_cap);
  const unsigned long long kp = ctl->key_prefix;   // key bits above this digit
  const unsigned long long ip = ctl->idx_prefix;
  const unsigned tau = ctl->tau_key;
  for (unsigned long long c = (unsigned long long)blockIdx.x * SEL_THREADS + tid; c < ncand;
       c += (unsigned long long)gridDim.x * SEL_THREADS) {
    unsigned key = a.cand_key[c];
    if (round < 3) {
      if (round > 0 && (key >> (shift + bits)) != kp) continue;
      atomicAdd(&h[(key >> shift) & ((1u << bits) - 1)], 1u);
    } else {
      if (key != tau) continue;
      unsigned long long idx = (unsigned long long)a.cand_idx[c];
      if ((idx >> (shift + bits)) != ip) continue;
      atomicAdd(&h[(idx >> shift) & ((1ull << bits) - 1)], 1u);
    }
  }
  __syncthreads();
  for (int b = tid; b < (1 << bits); b += SEL_THREADS)
    if (h[b]) atomicAdd(&ctl->sel_hist[b], h[b]);
  __threadfence();
  __shared__ unsigned s_last;
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&ctl->done_ctas, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: copy the global histogram, clear it, find the digit
  for (int b = tid; b < kHistBins; b += SEL_THREADS) {
    h[b] = (b < (1 << bits)) ? atomicExch(&ctl->sel_hist[b], 0u) : 0u;
  }
  __syncthreads();
  // find bin (single warp-free approach: each thread scans a slice)
  __shared__ int s_bin;
  __shared__ unsigned long long s_before;
  __shared__ unsigned s_in;
  const int nb = 1 << bits;
  const bool from_top = round < 3;
  const unsigned long long need = (unsigned long long)ctl->need;
  const int per = (nb + SEL_THREADS - 1) / SEL_THREADS;
  unsigned loc = 0;
  for (int o = tid * per; o < min(nb, tid * per + per); ++o) loc += h[from_top ? nb - 1 - o : o];
  unsigned tot;
  unsigned excl = block_excl_scan(loc, &tot);
  if (tid == 0) s_bin = -1;
  __syncthreads();
  unsigned long long run = excl;
  for (int o = tid * per; o < min(nb, tid * per + per); ++o) {
    int b = from_top ? nb - 1 - o : o;
    unsigned c = h[b];
    if (run < need && run + c >= need) { s_bin = b; s_before = run; s_in = c; }
    run += c;
  }
  __syncthreads();
  if (tid == 0) {
    ctl->done_ctas = 0u;
    const int b = s_bin;
    if (b < 0) {            // inconsistent counts: cannot happen for valid candidates
      ctl->abort = 1;
      ctl->need_bigger_cand = 1;
    } else if (round < 3) {
      ctl->key_prefix = (kp << bits) | (unsigned)b;
      ctl->need = (long long)(need - s_before);
      if (round == 2) {
        ctl->tau_key = (unsigned)ctl->key_prefix;
        ctl->key_done = 1;
        if ((unsigned long long)ctl->need == s_in) {   // every tie is taken
          ctl->idx_cut = ~0ull;
          ctl->idx_done = 1;
        }
      }
    } else {
      ctl->idx_prefix = (ip << bits) | (unsigned)b;
      ctl->need = (long long)(need - s_before);
      if (round == 6) {
        ctl->idx_cut = ctl->idx_prefix;
        ctl->idx_done = 1;
      }
    }
  }
}

// --------------------------------------------------------------------------------------
// Emit S_t, objective, and next-iteration bookkeeping (last block).
// --------------------------------------------------------------------------------------
constexpr int EMIT_THREADS = 256, EMIT_ITEMS = 8;

__global__ void __launch_bounds__(EMIT_THREADS)
k_emit(EmitArgs a) {
  Ctl* ctl = a.ctl;
  if (ctl->abort || !ctl->ready) return;
  const int tid = threadIdx.x;
  const int nb = ctl->cur ^ 1;
  const unsigned long long ncand = (ctl->need > 0) ? min(ctl->cand_count, a.cand_cap) : 0ull;
  const unsigned tau = ctl->tau_key;
  const unsigned long long cut = ctl->idx_cut;
  long long* Sidx = a.S_idx[nb];
  float* Sval = a.S_val[nb];
  unsigned* bits = a.sbits ? a.sbits + (size_t)nb * (size_t)a.sbits_words : nullptr;   // clear until now
  double dsum = 0.0;
  const unsigned long long tile = (unsigned long long)EMIT_THREADS * EMIT_ITEMS;
  __shared__ unsigned long long s_base;
  for (unsigned long long t0 = (unsigned long long)blockIdx.x * tile; t0 < ncand;
       t0 += (unsigned long long)gridDim.x * tile) {
    unsigned sel = 0;
    unsigned cnt = 0;
#pragma unroll
    for (int j = 0; j < EMIT_ITEMS; ++j) {
      unsigned long long c = t0 + (unsigned long long)j * EMIT_THREADS + tid;
      if (c < ncand) {
        unsigned key = a.cand_key[c];
        bool s = key > tau || (key == tau && (unsigned long long)a.cand_idx[c] <= cut);
        if (s) { sel |= 1u << j; ++cnt; }
        else { float v = a.cand_val[c]; dsum += (double)v * (double)v; }
      }
    }
    unsigned total;
    unsigned off = block_excl_scan(cnt, &total);
    if (tid == 0) s_base = total ? atomicAdd(&ctl->nnz_new, (unsigned long long)total) : 0ull;
    __syncthreads();
    unsigned long long pos = s_base + off;
#pragma unroll
    for (int j = 0; j < EMIT_ITEMS; ++j) {
      if (sel & (1u << j)) {
        unsigned long long c = t0 + (unsigned long long)j * EMIT_THREADS + tid;
        if (pos < (unsigned long long)ctl->k_req) {   // never past the S buffers
          const long long idx = a.cand_idx[c];
          Sidx[pos] = idx;
          Sval[pos] = a.cand_val[c];
          if (bits) atomicOr(&bits[idx >> 5], 1u << (idx & 31));
        }
        ++pos;
      }
    }
  }
  double bs = block_sum_double(dsum);
  if (tid == 0 && bs != 0.0) atomicAdd(&ctl->sumsq_cand_out, bs);
  __threadfence();
  __shared__ unsigned s_last;
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&ctl->done_ctas2, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last || tid != 0) return;
  __threadfence();
  // ---- last thread of the last block: commit the iteration ----
  const double obj = atomicAdd(&ctl->sumsq_noncand, 0.0) + atomicAdd(&ctl->sumsq_cand_out, 0.0);
  ctl->obj = obj;
  ctl->rel_err = ctl->normX2 > 0.0 ? obj / ctl->normX2 : 0.0;
  ctl->nnz_prev = ctl->nnz_cur;
  {
    unsigned long long got = atomicAdd(&ctl->nnz_new, 0ull);
    if (got > (unsigned long long)ctl->k_eff) {   // selection inconsistent: keep the old S
      ctl->nnz_cur = ctl->nnz_prev;
      ctl->need_bigger_cand = 1;
      ctl->abort = 1;
      ctl->done_ctas2 = 0u;
      return;
    }
    ctl->nnz_cur = (long long)got;
  }
  ctl->cur = nb;
  ctl->iter += 1;
  ctl->slot_parity ^= 1;          // normalisers written during this iteration become current
  ctl->last_passes = ctl->passes_run;
  if (ctl->tol >= 0.0 && ctl->rel_err <= ctl->tol) {
    ctl->converged = 1;
    ctl->abort = 1;
  }
  // threshold guess for the next S-step: two digit-1 bins below the k-th key
  if (ctl->need > 0) {
    int b = (int)(ctl->tau_key >> kD1Shift) - 2;
    ctl->next_guess = b > 0 ? ((unsigned)b << kD1Shift) : 1u;
  } else {
    ctl->next_guess = 0u;
  }
  // reset per-iteration state
  ctl->done_ctas2 = 0u;
  ctl->nnz_new = 0ull;
  ctl->plan[0] = ctl->next_guess ? PASS_CAND : PASS_FULL;
  ctl->plan[1] = PASS_NONE;
  ctl->plan[2] = PASS_NONE;
  ctl->guess[0] = ctl->next_guess;
  ctl->ready = 0;
  ctl->cand_count = 0ull;
  ctl->sumsq_noncand = 0.0;
  ctl->sumsq_full = 0.0;
  ctl->sumsq_cand_out = 0.0;
  ctl->k_eff = ctl->k_req;
  ctl->key_prefix = 0ull;
  ctl->idx_prefix = 0ull;
  ctl->key_done = 0;
  ctl->idx_done = 0;
  ctl->tau_key = 0u;
  ctl->idx_cut = 0ull;
  ctl->need = 0;
}

// Z := X on the entries of S_{t-1}, then Z := X - S_t on the entries of S_t.
// Z and Zt hold (X - S) zscale[0].  An entry whose scaled magnitude reaches kZRange
// flags range_err; the next product sees the flag, abandons that iteration before
// reading Z, and the caller rescales Z (setting abort here would cut this update short
// in blocks that have not started yet).
__device__ __forceinline__ void z_write(const EmitArgs& a, long long i, long long j, float z, float zs, bool& bad) {
  const float v = z * zs;
  bad |= fabsf(v) >= kZRange && isfinite(v);
  a.Z[i * a.ldz + j] = v;
  if (a.Zt) a.Zt[j * a.ldzt + i] = v;
  if (a.Z16) reinterpret_cast<__half*>(a.Z16)[i * a.ldz + j] = __float2half_rn(v);     // precision form's copies
  if (a.Zt16) reinterpret_cast<__half*>(a.Zt16)[j * a.ldzt + i] = __float2half_rn(v);
}

__device__ __forceinline__ void z_flag(Ctl* ctl, bool bad) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) ctl->range_err = 1;
}

// Row and column of a linear index (idx = i n + j): a float estimate of the quotient,
// refined once from the remainder and then corrected exactly in integers (no 64-bit
// division; the estimate is off by at most a couple of units for any size).
__device__ __forceinline__ void split_idx(long long idx, long long n, float ninv, long long& i, long long& j) {
  long long q = (long long)((float)idx * ninv);
  long long r = idx - q * n;
  q += (long long)((float)r * ninv);
  r = idx - q * n;
  while (r < 0) {
    --q;
    r += n;
  }
  while (r >= n) {
    ++q;
    r -= n;
  }
  i = q;
  j = r;
}

// One entry per thread (the grid covers the largest possible support, k).  The update
// also runs after the iteration that met the stop test (converged sets abort only to
// stop the iterations after it), so Z always matches the committed S.
__device__ __forceinline__ bool z_skip(const Ctl* ctl) { return ctl->abort && !ctl->converged; }

// The update of Z (and its copies) from S_{t-1} to S_t, one launch: entries of Omega_{t-1}
// that left the support get Z = X back, and Z = X - S_t on Omega_t.  The two sets are
// disjoint (the restore skips every entry the emit marked in the bitmap of Omega_t), so
// thread e does entry e of both lists.  The bitmap of Omega_{t-1} is cleared on the way
// (every set bit of it belongs to an entry of Omega_{t-1}, so each such entry simply
// zeroes its word).
__global__ void k_z_update(EmitArgs a) {
  Ctl* ctl = a.ctl;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (z_skip(ctl)) return;
  const long long np = ctl->nnz_prev, nc = ctl->nnz_cur;
  if ((long long)blockIdx.x * blockDim.x >= (np > nc ? np : nc)) return;
  const float zs = a.zscale ? a.zscale[0] : 1.f;
  const float ninv = 1.f / (float)a.n;
  const int cb = ctl->cur;
  bool bad = false;
  if (e < np) {
    const long long idx = a.S_idx[cb ^ 1][e];
    const unsigned* now = a.sbits ? a.sbits + (size_t)cb * (size_t)a.sbits_words : nullptr;
    if (!now || !((__ldcg(&now[idx >> 5]) >> (idx & 31)) & 1u)) {
      long long i, j;
      split_idx(idx, a.n, ninv, i, j);
      z_write(a, i, j, a.X[i * a.ldx + j], zs, bad);
    }
    if (a.sbits) a.sbits[(size_t)(cb ^ 1) * (size_t)a.sbits_words + (size_t)(idx >> 5)] = 0u;
  }
  if (e < nc) {
    const long long idx = a.S_idx[cb][e];
    long long i, j;
    split_idx(idx, a.n, ninv, i, j);
    z_write(a, i, j, a.X[i * a.ldx + j] - a.S_val[cb][e], zs, bad);
  }
  z_flag(ctl, bad);
}

// The support bitmap of the committed S (bitmap ctl->cur) from its index list, one entry
// per thread; both bitmaps were cleared before (after an S-step cut short).
__global__ void k_sbits_rebuild(unsigned* sbits, long long words, long long* S0, long long* S1, const Ctl* ctl) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cb = ctl->cur;
  if (e >= ctl->nnz_cur) return;
  const long long idx = (cb ? S1 : S0)[e];
  atomicOr(&sbits[(size_t)cb * (size_t)words + (size_t)(idx >> 5)], 1u << (idx & 31));
}

// Per-iteration S-step state back to "start of an iteration" (one thread).
__global__ void k_reset_iter(Ctl* ctl) {
  for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) {
    ctl->hist[b] = 0u;
    ctl->sel_hist[b] = 0u;
  }
  if (threadIdx.x != 0) return;
  ctl->plan[0] = ctl->next_guess ? PASS_CAND : PASS_FULL;
  ctl->plan[1] = PASS_NONE;
  ctl->plan[2] = PASS_NONE;
  ctl->guess[0] = ctl->next_guess;
  ctl->guess[1] = ctl->guess[2] = 0u;
  ctl->passes_run = 0;
  ctl->ready = 0;
  ctl->need_bigger_cand = 0;
  ctl->cand_count = 0ull;
  ctl->k_eff = ctl->k_req;
  ctl->sumsq_noncand = ctl->sumsq_full = ctl->sumsq_cand_out = 0.0;
  ctl->done_ctas = ctl->done_ctas2 = 0u;
  ctl->key_prefix = ctl->idx_prefix = 0ull;
  ctl->need = 0;
  ctl->tau_key = 0u;
  ctl->key_done = ctl->idx_done = 0;
  ctl->idx_cut = 0ull;
  ctl->nnz_new = 0ull;
  ctl->rank_drop = 0;
  ctl->abort = 0;
  ctl->nonfinite = 0;
  ctl->chol_fail = 0;
  ctl->converged = 0;
  ctl->alarm = 0;
  ctl->timeout = 0;
}

}  // namespace

cudaError_t prepare_select_kernels() {
  return cudaFuncSetAttribute(k_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResSmem);
}

void launch_reset_iter(Ctl* ctl, cudaStream_t st) { k_reset_iter<<<1, 256, 0, st>>>(ctl); }

void launch_residual(const ResidualArgs& a, int nsm, cudaStream_t st) {
  const int64_t ntiles = ((a.m + RT_M - 1) / RT_M) * ((a.n + RT_N - 1) / RT_N);
  int64_t grid = 3LL * nsm;
  if (grid > ntiles) grid = ntiles;
  k_residual<<<(unsigned)grid, RES_THREADS, kResSmem, st>>>(a);
}

void launch_after_pass(Ctl* ctl, int pass, long long k, unsigned long long cap, cudaStream_t st) {
  k_after_pass<<<1, CTL_THREADS, 0, st>>>(ctl, pass, k, cap);
}

void launch_select_round(const SelectArgs& a, int nsm, cudaStream_t st) {
  k_select_round<<<(unsigned)(2 * nsm), SEL_THREADS, 0, st>>>(a);
}

void launch_emit(const EmitArgs& a, int nsm, cudaStream_t st) {
  k_emit<<<(unsigned)(2 * nsm), EMIT_THREADS, 0, st>>>(a);
}

void launch_sbits_rebuild(unsigned* sbits, long long words, long long* const S_idx[2], const Ctl* ctl,
                          long long max_nnz, cudaStream_t st) {
  const long long nb = (max_nnz + 255) / 256;
  k_sbits_rebuild<<<(unsigned)(nb > 0 ? nb : 1), 256, 0, st>>>(sbits, words, S_idx[0], S_idx[1], ctl);
}

void launch_z_update(const EmitArgs& a, int nsm, cudaStream_t st) {
  (void)nsm;
  const long long nb = (a.max_nnz + 255) / 256;
  const unsigned grid = (unsigned)(nb > 0 ? nb : 1);
  k_z_update<<<grid, 256, 0, st>>>(a);
}

}  // namespace godec
