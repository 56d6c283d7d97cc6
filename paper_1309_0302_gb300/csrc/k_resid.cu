// Residual pass of the S-step on the tensor cores (Algorithm 1, eq. raw_lss).
//
//   R = X - L,   L = U diag(sigma) V^T = (A B^T) / s_Z,
//   A = U diag(sqrt(sigma s_Z)),  B = V diag(sqrt(sigma s_Z))
//
// A and B (m x RP, n x RP) are split once per iteration into two float16 terms each
// (x = h + 2^-11 l, h cut to 11 significant bits, l rounded), stored as rows of 128
// halves: 64 of h (K zero-padded to 64) then 64 of l.  Per 128 x 64 tile of R:
//   D[:, 0:128]  = A_h [B_h; B_l]^T      (N = 128, K = 64)
//   D[:, 64:128] += A_l B_h^T           (N = 64)
// so L = (D[:, :64] + 2^-11 D[:, 64:]) / s_Z to float32 accuracy (the dropped A_l B_l
// term is 2^-22 relative).  s_Z, the scale of the working copy of X - S, bounds
// sigma s_Z and keeps A and B inside the float16 range.
//
// The epilogue forms R from the accumulator and the X tile (TMA-staged), and does
// what k_residual does: a 4096-bin histogram of the top key bits (full mode) or the
// candidates with key >= guess (candidate mode), the float64 sums of R^2, and the
// non-finite check.  A dump mode writes R densely (testing).  Candidates are staged
// per warp in shared memory (the histogram's space) and written out with one global
// atomic per full buffer, so no tile waits on a contended atomic.
//
// Warps: 0 TMA producer of the X tiles, 18 TMA producer of the B and A tiles (the MMA's
// operands), 1 MMA issuer and TMEM owner, 2-17 epilogue (four per TMEM lane quarter, one
// per 16-column quarter of the tile).  With one producer for everything, B(t) (from L2,
// ~2 us under the stream) was issued only once X(t-1) had a free slot, and the chain
// epilogue(t-4) -> B(t) -> MMA(t) -> epilogue(t) set the pace at about half the memory
// rate; with B and A on their own producer and three B slots, the MMAs run ahead and
// the X ring alone paces the pass.  Tiles
// are taken in row-band order in one contiguous range per CTA, so A changes at most
// a few times per CTA.  Every wait is bounded; a timeout sets ctl->timeout.
#include <cuda.h>
#include <cuda_fp16.h>

#include "godec_internal.cuh"
#include "tc_util.cuh"

namespace godec {

namespace {

using namespace tc;

constexpr int RM = 128, RNC = 64;           // tile rows and columns
constexpr int NXS = 4, NBS = 3;             // X slots, B slots (B tiles come from L2)
constexpr int kAcc = 4;                     // accumulators in TMEM (128 columns each)
constexpr int kEpiW = 16;
constexpr int kECols = RNC / (kEpiW / 4);   // columns of a tile per epilogue thread
constexpr int kRThreads = 32 * (3 + kEpiW);
constexpr int kBWarp = 2 + kEpiW;           // the B / A producer
constexpr size_t kXBox = (size_t)RM * 32 * 4;     // 32 float32 columns x 128 rows = 16 KB
constexpr size_t kXSlot = 2 * kXBox;
constexpr size_t kBBox = (size_t)RNC * 128;       // 64 halves x 64 rows = 8 KB
constexpr size_t kBSlot = 2 * kBBox;              // [B_h; B_l] = 128 rows
constexpr size_t kAHalf = (size_t)RM * 128;       // 64 halves x 128 rows = 16 KB
constexpr size_t kOffX = 0;
constexpr size_t kOffB = kOffX + NXS * kXSlot;
constexpr size_t kOffA = kOffB + NBS * kBSlot;
constexpr size_t kOffH = kOffA + 2 * kAHalf;
constexpr size_t kRSmem = kOffH + (size_t)kHistBins * 4 + 1024;
constexpr uint32_t kRWait = 1u << 20;
constexpr float kLoInv = 1.f / 2048.f;
constexpr int kStage = 64;                        // staged candidates per epilogue warp
static_assert(kEpiW * kStage * 16 <= kHistBins * 4, "candidate staging fits the histogram space");
static_assert(kRSmem <= 232448 - 1024, "shared memory of the residual pass");

struct RTArgs {
  int64_t m, n;
  int pass;
  Ctl* ctl;
  unsigned* cand_key;
  long long* cand_idx;
  float* cand_val;
  unsigned long long cand_cap;
  const float* zscale;      // zscale[1] = 1 / s_Z
  float* dump;              // dump mode when non-null: R into dump (row stride ldd)
  int64_t ldd;
};

__device__ __forceinline__ unsigned rkey(float v) { return __float_as_uint(v) & 0x7fffffffu; }

// r[q] for a run-time q < 16 by a select tree on q's bits: the values stay in registers
// (an indexed access would put the array in local memory)
__device__ __forceinline__ float pick16(const float (&r)[16], int q) {
  float a8[8], a4[4], a2[2];
#pragma unroll
  for (int i = 0; i < 8; ++i) a8[i] = (q & 8) ? r[i + 8] : r[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) a4[i] = (q & 4) ? a8[i + 4] : a8[i];
#pragma unroll
  for (int i = 0; i < 2; ++i) a2[i] = (q & 2) ? a4[i + 2] : a4[i];
  return (q & 1) ? a2[1] : a2[0];
}

__device__ __forceinline__ bool wwait(uint64_t* bar, uint32_t parity, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, kRWait) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

__device__ __forceinline__ void rtimeout(Ctl* ctl, volatile int* s_err) {
  *s_err = 1;
  ctl->timeout = 1;
  ctl->abort = 1;
}

__global__ void __launch_bounds__(kRThreads, 1)
k_resid_tc(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapA,
           const __grid_constant__ CUtensorMap mapB, RTArgs a) {
  Ctl* ctl = a.ctl;
  __shared__ int s_mode;
  __shared__ unsigned s_guess;
  if (threadIdx.x == 0) {
    int md = PASS_NONE;
    if (a.dump) md = PASS_DUMP;
    else if (!ctl->abort) md = ctl->plan[a.pass];
    s_mode = md;
    s_guess = (md == PASS_CAND) ? ctl->guess[a.pass] : 0u;
  }
  __syncthreads();
  const int mode = s_mode;
  if (mode == PASS_NONE) return;   // uniform: every thread read the same flag
  const unsigned guess = s_guess;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sX = sm + kOffX;
  unsigned char* sB = sm + kOffB;
  unsigned char* sA = sm + kOffA;
  unsigned* hist = reinterpret_cast<unsigned*>(sm + kOffH);
  __shared__ uint64_t xfull[NXS], xempty[NXS], bfull[NBS], bempty[NBS], afull, aempty, accfull[kAcc],
      accempty[kAcc], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_err;
  __shared__ double s_red[kEpiW];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m = a.m, n = a.n;
  const int64_t nbj = (n + RNC - 1) / RNC, nbi = (m + RM - 1) / RM, T = nbi * nbj;
  const int G = gridDim.x, c = blockIdx.x;
  const int64_t g0 = (int64_t)c * T / G, g1 = (int64_t)(c + 1) * T / G;
  if (tid == 0) {
    for (int s = 0; s < NXS; ++s) {
      mbar_init(&xfull[s], 1);
      mbar_init(&xempty[s], kEpiW);
    }
    for (int s = 0; s < NBS; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    mbar_init(&afull, 1);
    mbar_init(&aempty, 1);
    for (int b = 0; b < kAcc; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], kEpiW);
    }
    mbar_init(&mma_done, 1);
    fence_barrier_init();
    s_err = 0;
  }
  if (mode == PASS_FULL)
    for (int b = tid; b < kHistBins; b += kRThreads) hist[b] = 0u;
  if (warp == 1) tmem_alloc(&tmem_base, 128 * kAcc);
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer: X tiles ----------------
    if (lane == 0) {
      int64_t ib = g0 / nbj, jb = g0 % nbj;
      int sx = 0;
      uint32_t phx = 0;
      int64_t nx = 0;
      const uint64_t pol = policy_evict_first();
      for (int64_t g = g0; g < g1 && !s_err; ++g) {
        if (!mbar_wait(&xempty[sx], phx ^ 1u, kRWait)) { rtimeout(ctl, &s_err); break; }
        // both boxes always: columns past n (and rows past m) are zero-filled, and so are
        // the rows of A and B past m and n, which makes R exactly 0 there
        mbar_expect_tx(&xfull[sx], (uint32_t)(2 * kXBox));
        // X is streamed once per pass and is larger than L2: evict its lines first
        tma_load_2d_hint(sX + sx * kXSlot, &mapX, &xfull[sx], (int)(jb * RNC), (int)(ib * RM), pol);
        tma_load_2d_hint(sX + sx * kXSlot + kXBox, &mapX, &xfull[sx], (int)(jb * RNC + 32), (int)(ib * RM), pol);
        ++nx;
        if (++sx == NXS) { sx = 0; phx ^= 1u; }
        if (++jb == nbj) { jb = 0; ++ib; }
      }
      // every copy issued has landed before the CTA may exit
      for (int64_t j = (nx > NXS ? nx - NXS : 0); j < nx; ++j)
        if (!mbar_wait(&xfull[(int)(j % NXS)], (uint32_t)((j / NXS) & 1), kRWait)) rtimeout(ctl, &s_err);
    }
  } else if (warp == kBWarp) {
    // ---------------- TMA producer: B tiles and the A band ----------------
    if (lane == 0) {
      int64_t band = -1, ib = g0 / nbj, jb = g0 % nbj;
      int nband = 0, sb = 0;
      uint32_t phb = 0;
      int64_t nbb = 0;
      for (int64_t g = g0; g < g1 && !s_err; ++g) {
        if (ib != band) {
          if (nband > 0 && !mbar_wait(&aempty, (uint32_t)((nband - 1) & 1), kRWait)) { rtimeout(ctl, &s_err); break; }
          mbar_expect_tx(&afull, (uint32_t)(2 * kAHalf));
          tma_load_2d(sA, &mapA, &afull, 0, (int)(ib * RM));
          tma_load_2d(sA + kAHalf, &mapA, &afull, 64, (int)(ib * RM));
          band = ib;
          ++nband;
        }
        if (!mbar_wait(&bempty[sb], phb ^ 1u, kRWait)) { rtimeout(ctl, &s_err); break; }
        mbar_expect_tx(&bfull[sb], (uint32_t)kBSlot);
        tma_load_2d(sB + sb * kBSlot, &mapB, &bfull[sb], 0, (int)(jb * RNC));
        tma_load_2d(sB + sb * kBSlot + kBBox, &mapB, &bfull[sb], 64, (int)(jb * RNC));
        ++nbb;
        if (++sb == NBS) { sb = 0; phb ^= 1u; }
        if (++jb == nbj) { jb = 0; ++ib; }
      }
      for (int64_t j = (nbb > NBS ? nbb - NBS : 0); j < nbb; ++j)
        if (!mbar_wait(&bfull[(int)(j % NBS)], (uint32_t)((j / NBS) & 1), kRWait)) rtimeout(ctl, &s_err);
      if (nband > 0 && !mbar_wait(&afull, (uint32_t)((nband - 1) & 1), kRWait)) rtimeout(ctl, &s_err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id_hi = idesc_f16(RM, 128), id_lo = idesc_f16(RM, 64);
      int64_t jb = g0 % nbj;
      bool new_band = true;
      int nb = 0, sb = 0, ai = 0;
      uint32_t phb = 0;
      for (int64_t g = g0; g < g1 && !s_err; ++g) {
        if (new_band) {
          if (!mbar_wait(&afull, (uint32_t)(nb & 1), kRWait)) { rtimeout(ctl, &s_err); break; }
          ++nb;
        }
        const int b = ai % kAcc;
        if (!mbar_wait(&bfull[sb], phb, kRWait) ||
            !mbar_wait(&accempty[b], (uint32_t)(((ai / kAcc) & 1) ^ 1), kRWait)) {
          rtimeout(ctl, &s_err);
          break;
        }
        tc_fence_after();
        const uint32_t dcol = tbase + (uint32_t)(b * 128);
        const uint64_t dah = sdesc_k128(sA), dal = sdesc_k128(sA + kAHalf), db = sdesc_k128(sB + sb * kBSlot);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t off = (uint64_t)((kk * 16 * 2) >> 4);   // 32 bytes per 16-wide K step
          mma_bf16(dcol, dah + off, db + off, id_hi, kk > 0 ? 1u : 0u);
          mma_bf16(dcol + 64, dal + off, db + off, id_lo, 1u);
        }
        mma_commit(&bempty[sb]);
        mma_commit(&accfull[b]);
        new_band = ++jb == nbj;
        if (new_band) jb = 0;
        if (g + 1 == g1 || new_band) mma_commit(&aempty);
        if (++sb == NBS) { sb = 0; phb ^= 1u; }
        ++ai;
      }
      mma_commit(&mma_done);
      if (!mbar_wait(&mma_done, 0, kRWait)) rtimeout(ctl, &s_err);
    }
  } else {
    // ---------------- epilogue ----------------
    // Each thread owns one row and 32 columns of the tile: R = X - (D_h + 2^-11 D_l) / s_Z,
    // formed with two FMAs (1 / s_Z is a power of two, so the scaled terms are exact).
    const int w = warp - 2;
    const int q4 = warp & 3, cq = w >> 2;   // TMEM lane quarter; column quarter of the tile
    const int row = q4 * 32 + lane, sw = row & 7;
    const int f4b = (cq & 1) * 4;           // this quarter's first float4 in its 128-byte box row
    const uint32_t tlane = (uint32_t)(q4 * 32) << 16;
    const float zinv = a.zscale[1], zlo = zinv * kLoInv;
    // candidate iff key >= max(guess, 1); for a non-NaN value that is |R| >= gf (a NaN
    // fails the compare, lands in the sum and is caught there)
    const float gf = __uint_as_float(guess > 1u ? guess : 1u);
    int64_t ib = g0 / nbj, jb = g0 % nbj;
    int sx = 0, ai = 0;
    uint32_t phx = 0;
    // sum of R^2 over the non-candidates: float per tile, compensated (Kahan) across tiles,
    // float64 once at the end (a float64 add per tile and thread kept GB300's slow
    // float64 pipe busy and stalled the epilogue)
    float ssum = 0.f, scmp = 0.f;
    bool bad = false;
    // this warp's candidate staging area (candidate mode uses the histogram's space)
    unsigned* st_key = reinterpret_cast<unsigned*>(hist) + w * kStage;
    float* st_val = reinterpret_cast<float*>(hist) + kEpiW * kStage + w * kStage;
    long long* st_idx = reinterpret_cast<long long*>(reinterpret_cast<float*>(hist) + 2 * kEpiW * kStage) + w * kStage;
    int staged = 0;
    auto flush = [&]() {
      if (staged == 0) return;
      unsigned long long base = 0ull;
      if (lane == 0) base = atomicAdd(&ctl->cand_count, (unsigned long long)staged);
      base = __shfl_sync(0xffffffffu, base, 0);
      __syncwarp();
      for (int e = lane; e < staged; e += 32)
        if (base + e < a.cand_cap) {
          a.cand_key[base + e] = st_key[e];
          a.cand_idx[base + e] = st_idx[e];
          a.cand_val[base + e] = st_val[e];
        }
      __syncwarp();
      staged = 0;
    };
    for (int64_t g = g0; g < g1; ++g) {
      if (__any_sync(0xffffffffu, s_err != 0)) break;
      const int b = ai % kAcc;
      if (!wwait(&accfull[b], (uint32_t)((ai / kAcc) & 1), lane) || !wwait(&xfull[sx], phx, lane)) {
        if (lane == 0) rtimeout(ctl, &s_err);
        break;
      }
      tc_fence_after();
      const uint32_t taddr = tbase + (uint32_t)(b * 128) + tlane + (uint32_t)(cq * kECols);
      float vh[kECols], vl[kECols];
      tmem_ld16x2(taddr, taddr + 64, vh, vl);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[b]);
      float4* xs = reinterpret_cast<float4*>(sX + sx * kXSlot + (cq >> 1) * kXBox + row * 128);
      float f0 = 0.f, f1 = 0.f;
      if (mode == PASS_CAND) {
        // R in registers, the candidate columns as a mask; branch-free: the candidate bit
        // by select, the non-candidate square by a selected factor (a NaN fails the
        // compare and reaches the sum)
        static_assert(kECols == 16, "pick16");
        float rr[kECols];
        unsigned cm = 0u;
#pragma unroll
        for (int u = 0; u < kECols / 4; ++u) {
          const float4 x = xs[(f4b + u) ^ sw];
          const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = 4 * u + e;
            rr[q] = fmaf(-vl[q], zlo, fmaf(-vh[q], zinv, xv[e]));
            const bool cand = fabsf(rr[q]) >= gf;
            cm |= cand ? (1u << q) : 0u;
            const float w2 = cand ? 0.f : rr[q];
            if (e & 1) f1 = fmaf(w2, rr[q], f1);
            else f0 = fmaf(w2, rr[q], f0);
          }
        }
        if (!isfinite(f0 + f1))   // rare: tell a NaN or an infinity from an overflowing sum
#pragma unroll
          for (int q = 0; q < kECols; ++q) bad |= rkey(rr[q]) >= 0x7f800000u;
        // the candidates, one per lane and round, in lane order
        const int tot = (int)__reduce_add_sync(0xffffffffu, (unsigned)__popc(cm));
        if (tot) {
          if (staged + tot > kStage) flush();
          unsigned* dk = st_key + staged;
          long long* di = st_idx + staged;
          float* dv = st_val + staged;
          unsigned long long lim = (unsigned long long)kStage;
          if (tot > kStage) {   // more than a buffer in one tile: straight out
            unsigned long long base = 0ull;
            if (lane == 0) base = atomicAdd(&ctl->cand_count, (unsigned long long)tot);
            base = __shfl_sync(0xffffffffu, base, 0);
            dk = a.cand_key + base;
            di = a.cand_idx + base;
            dv = a.cand_val + base;
            lim = a.cand_cap > base ? a.cand_cap - base : 0ull;
          }
          const long long rb = (long long)((ib * RM + row) * n + jb * RNC + cq * kECols);
          const unsigned lt_mask = (1u << lane) - 1u;
          unsigned pos = 0u, mm = cm;
          unsigned bal = __ballot_sync(0xffffffffu, mm != 0u);
          while (bal) {
            if (mm) {
              const int q = __ffs(mm) - 1;
              mm &= mm - 1u;
              const unsigned p = pos + __popc(bal & lt_mask);
              const float v = pick16(rr, q);
              const unsigned key = rkey(v);
              bad |= key >= 0x7f800000u;
              if (p < lim) {
                dk[p] = key;
                di[p] = rb + q;
                dv[p] = v;
              }
            }
            pos += (unsigned)__popc(bal);
            bal = __ballot_sync(0xffffffffu, mm != 0u);
          }
          __syncwarp();
          if (tot <= kStage) staged += tot;
        }
      } else if (mode == PASS_FULL) {
#pragma unroll
        for (int u = 0; u < kECols / 4; ++u) {
          const float4 x = xs[(f4b + u) ^ sw];
          const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = 4 * u + e;
            const float r = fmaf(-vl[q], zlo, fmaf(-vh[q], zinv, xv[e]));
            const unsigned key = rkey(r);
            bad |= key >= 0x7f800000u;
            if (e & 1) f1 = fmaf(r, r, f1);
            else f0 = fmaf(r, r, f0);
            if (key) atomicAdd(&hist[key >> kD1Shift], 1u);
          }
        }
      } else {   // dump
        const int64_t i = ib * RM + row, j0 = jb * RNC + cq * kECols;
#pragma unroll
        for (int u = 0; u < kECols / 4; ++u) {
          const float4 x = xs[(f4b + u) ^ sw];
          const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = 4 * u + e;
            if (i < m && j0 + q < n) a.dump[i * a.ldd + j0 + q] = fmaf(-vl[q], zlo, fmaf(-vh[q], zinv, xv[e]));
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&xempty[sx]);
      if (++sx == NXS) { sx = 0; phx ^= 1u; }
      ++ai;
      if (++jb == nbj) { jb = 0; ++ib; }
      const float y = (f0 + f1) - scmp, t = ssum + y;
      scmp = (t - ssum) - y;
      ssum = t;
    }
    double dsum = (double)ssum - (double)scmp;
    if (mode == PASS_CAND) flush();
    // sums over the epilogue warps, then one atomic per CTA
#pragma unroll
    for (int o = 16; o; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if (lane == 0) s_red[w] = dsum;
    if (__any_sync(0xffffffffu, bad) && lane == 0) ctl->nonfinite = 1;
    named_sync(1, 32 * kEpiW);
    if (w == 0 && lane == 0 && mode != PASS_DUMP) {
      double t = 0.0;
      for (int k = 0; k < kEpiW; ++k) t += s_red[k];
      atomicAdd(mode == PASS_FULL ? &ctl->sumsq_full : &ctl->sumsq_noncand, t);
    }
    if (mode == PASS_FULL)
      for (int bb = w * 32 + lane; bb < kHistBins; bb += 32 * kEpiW)
        if (hist[bb]) atomicAdd(&ctl->hist[bb], hist[bb]);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 128 * kAcc);
  }
}

// Rows of A (i < m) and B (i >= m): 64 halves of h (K padded to 64), then 64 of l.
__global__ void k_lsplit(const float* __restrict__ U, const float* __restrict__ V, const float* __restrict__ sigma,
                         int64_t m, int64_t n, int RP, int r, const float* __restrict__ zscale,
                         __half* __restrict__ A, __half* __restrict__ B, const int* skip) {
  if (block_skip(skip)) return;
  __shared__ float sq[64];
  if (threadIdx.x < 64) {
    const float s = threadIdx.x < r ? sigma[threadIdx.x] * zscale[0] : 0.f;
    sq[threadIdx.x] = s > 0.f ? sqrtf(s) : 0.f;
  }
  __syncthreads();
  // one warp per row, lane l for the column pair (2l, 2l+1): loads and both 64-byte halves
  // of the output row are written by coalesced warp-wide accesses
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < m + n; t += nwarps) {
    const bool isU = t < m;
    const int64_t i = isU ? t : t - m;
    const float* src = (isU ? U : V) + i * RP;
    __half2* dst = reinterpret_cast<__half2*>((isU ? A : B) + i * 128);
    const int l = 2 * lane;
    float v[2], h[2], lo[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      v[e] = (l + e < r) ? src[l + e] * sq[l + e] : 0.f;
      h[e] = __uint_as_float(__float_as_uint(v[e]) & 0xFFFFE000u);
      lo[e] = (v[e] - h[e]) * 2048.f;
    }
    dst[lane] = __floats2half2_rn(h[0], h[1]);
    dst[32 + lane] = __floats2half2_rn(lo[0], lo[1]);
  }
}

}  // namespace

cudaError_t prepare_resid_kernels() {
  return cudaFuncSetAttribute(k_resid_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmem);
}

void launch_lsplit(const float* U, const float* V, const float* sigma, int64_t m, int64_t n, int RP, int r,
                   const float* zscale, void* A, void* B, cudaStream_t st, const int* skip) {
  const int64_t tot = m + n;   // rows, one warp each, 8 warps a block, at most 4096 blocks
  int64_t blocks = (tot + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  k_lsplit<<<(unsigned)blocks, 256, 0, st>>>(U, V, sigma, m, n, RP, r, zscale,
                                                          reinterpret_cast<__half*>(A), reinterpret_cast<__half*>(B),
                                                          skip);
}

void launch_resid_tc(const ResidTcLaunch& l, cudaStream_t st) {
  RTArgs a;
  a.m = l.ra.m;
  a.n = l.ra.n;
  a.pass = l.ra.pass;
  a.ctl = l.ra.ctl;
  a.cand_key = l.ra.cand_key;
  a.cand_idx = l.ra.cand_idx;
  a.cand_val = l.ra.cand_val;
  a.cand_cap = l.ra.cand_cap;
  a.zscale = l.zscale;
  a.dump = l.dump;
  a.ldd = l.ldd;
  const int64_t T = ((a.m + RM - 1) / RM) * ((a.n + RNC - 1) / RNC);
  const int G = (int)(T < l.nsm ? T : l.nsm);
  k_resid_tc<<<G, kRThreads, kRSmem, st>>>(*reinterpret_cast<const CUtensorMap*>(l.mapX),
                                           *reinterpret_cast<const CUtensorMap*>(l.mapA),
                                           *reinterpret_cast<const CUtensorMap*>(l.mapB), a);
}

}  // namespace godec
