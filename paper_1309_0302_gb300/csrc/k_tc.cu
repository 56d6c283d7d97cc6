// Streaming product on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   part/out = Zsrc (rows x K, float32, row-major) * B (K x RP)   to float32 accuracy
//
// Two-term float16 split ("2xFP16"): with a power-of-two scale s_Z, each element is
// written x s_Z = h1 + 2^-11 h2, h1 = x s_Z cut to 11 significant bits (exact in
// float16), h2 = fp16((x s_Z - h1) 2^11) rounded to nearest; the
// skinny operand likewise, b s_B = c1 + 2^-11 c2, arrives already split and transposed
// as [c1^T; c2^T] (2 RP x K float16) from the step that produced it.  Then
//   x b s_Z s_B = h1 c1 + 2^-11 (h1 c2 + h2 c1) + O(2^-22),
// the dropped h2 c2 term being the only truncation.  Per 16-wide K step:
//   D[:, 0:2RP] += h1 [c1; c2]^T   and   D[:, RP:RP+RPl] += h2 (rows 0..RPl-1 of [c1; c2])^T,
// RPl = RP rounded up to 16 (the MMA's N granularity): columns RP..2RP-1 receive h2 c1,
// columns beyond 2RP collect a product nobody reads.  The result is
// (D[:, :RP] + 2^-11 D[:, RP:2RP]) / (s_Z s_B).  float16 MMAs run at twice the TF32
// rate with twice the K per instruction.
//
// A copier thread moves each landed 128 x 64 float32 tile of Zsrc from shared memory into
// tensor memory (tcgen05.cp) and frees the shared-memory slot when the copy completes;
// converter warps then turn the tile into the two packed float16 blocks (h1, h2) in place
// with TMEM loads and stores.  The working warps thus leave the shared-memory load path
// to the TMA stream.  Zsrc is either stored already scaled (the working copy of X - S,
// whose writers keep it inside the float16 range) or scaled here (a caller's matrix,
// scale from its exact maximum).
//
// Work split: the (128-row tile, 64-wide K stage) iteration space is cut into equal
// contiguous ranges, one per persistent CTA ("stream-K"), so every SM streams the same
// number of bytes whatever the tile count.  The tensor core accumulates a chunk of
// kChunk stages in TMEM (double-buffered); the 4 epilogue warps drain each chunk into
// float32 registers, so the tensor core's own accumulation never runs over more than
// kChunk * 64 terms (its additions are not round-to-nearest, and over thousands of
// terms of one sign the bias would show).  At a tile boundary the running sum goes to
// a partial slot.  The last segment of a tile to arrive adds the slots in order
// (deterministic), unscales, applies the normaliser T, and writes the rows, the next
// product's split transposed operand and the tile's Gram partial.
//
// Warps: 0 TMA producer of Zsrc tiles, 1 MMA issuer (and TMEM owner), 2-9 converters
// (two per TMEM lane quarter, one per 32-column half of the tile), 10-13 epilogue,
// 14 TMA producer of the skinny operand, 15 copier.
// TMEM (512 columns): 0-255 two accumulators of 128 columns, 256-447 three stage slots of
// 64 columns (the float32 tile, then per 32-column half 16 columns of packed h1 and 16
// of packed h2).
// Synchronisation per stage: TMA -> afull -> copier (after sfree) -> aempty (slot
// refilled) and cpdone -> converters -> tfull (after the skinny tile's bfull too) -> MMA
// -> sfree -> the stage slot and the skinny TMA slot.  The MMA issuer waits once and
// commits once per stage.
// Every wait is bounded; a timeout sets ctl->timeout and the CTA drains and exits.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "godec_internal.cuh"
#include "gram_tile.cuh"
#include "tc_util.cuh"

namespace godec {

namespace {

using namespace tc;

constexpr int BM = 128, BK = 64;   // rows per tile, K per stage (4 MMA steps of 16)
constexpr int NA = 5;              // shared-memory slots for Zsrc tiles (TMA ring)
constexpr int NS = 4;              // stage slots: skinny-operand tile in shared memory + converted
                                   // Zsrc tile in TMEM, freed together by one MMA commit
constexpr int kThreads = 512;
constexpr int kConvWarps = 8;
constexpr uint32_t kTmemCols = 512, kTA0 = 256, kTASlot = 64;
constexpr int EPI_LD = kMaxRP + 1;   // odd stride: row-wise and column-wise accesses are conflict-free
constexpr size_t kBoxA = (size_t)BM * 32 * 4;               // one 32-column float32 box, 16 KB
constexpr size_t kStageA = 2 * kBoxA;                       // 32 KB
constexpr size_t kStageB = (size_t)2 * kMaxRP * BK * 2;     // 16 KB (room for 2 x 64 rows of 64 halves)
constexpr size_t kOffA = 0;
constexpr size_t kOffB = kOffA + NA * kStageA;
// tile completion runs after the stream, in the then idle Zsrc ring
constexpr size_t kEpiBytes = (size_t)BM * EPI_LD * 4 + (size_t)kMaxRP * kMaxRP * 4;
constexpr size_t kTcSmem = kOffB + NS * kStageB + 1024;     // + alignment slack
static_assert(kEpiBytes <= NA * kStageA, "completion staging fits the Zsrc ring");
constexpr uint32_t kWaitLimit = 1u << 20;
constexpr float kLoScale = 2048.f, kLoInv = 1.f / 2048.f;
#ifndef GODEC_TC_CHUNK
#define GODEC_TC_CHUNK 2
#endif
constexpr int kChunk = GODEC_TC_CHUNK;   // K stages accumulated in TMEM before a drain
static_assert(kTcSmem <= 232448 - 1024, "shared memory of the tensor-core product");

struct TcArgs {
  int64_t rows, K;
  int RP;                   // columns kept (multiple of 8)
  int64_t ks, S;            // K stages per tile, total stages
  int G;                    // CTAs
  int maxseg;
  float* part;              // tiles x maxseg x BM x RP
  unsigned* counters;       // tiles
  float* out;               // rows x RP (nullable)
  __half* bt2;              // 2 RP x ldb split transposed output (nullable)
  int64_t ldb;
  const float* Tn0;
  const float* Tn1;
  const float* cscale;      // per-column output factor 1 / s_B (nullable: 1)
  const float* zscale;      // {s_Z, 1 / s_Z} (nullable: 1)
  int prescaled;            // Zsrc holds x s_Z already (s_Z then only undone in the epilogue)
  void* gram_part;
  int gram_mode;
  int t_upper;              // the normaliser is upper triangular
  int* pend;                // G x maxpend: tiles each CTA completes, deferred to its end
  int maxpend;
  int z_prefetch;           // Zsrc's first stages may be loaded before the programmatic wait
  Ctl* ctl;
};

__device__ __forceinline__ int64_t cta_of(int64_t g, int64_t S, int G) { return ((g + 1) * (int64_t)G - 1) / S; }

__device__ __forceinline__ void note_timeout(Ctl* ctl, volatile int* s_err) {
  *s_err = 1;
  if (ctl) {
    ctl->timeout = 1;
    ctl->abort = 1;
  }
}

// cvt.rn.f16x2: first source goes to the upper half, so element k sits in bits 0-15.
__device__ __forceinline__ uint32_t pack_h2(float even, float odd) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(odd), "f"(even));
  return d;
}

// Completion of tile t by its last segment, run by nthr threads (u = 0..nthr-1, a
// multiple of 32) that synchronise on named barrier `bar`: the partial slots are added
// in slot order (deterministic whoever finishes) and unscaled, the normaliser T applied,
// the rows and the next product's split transposed operand written, and the tile's Gram
// partial formed.  Ps (BM x EPI_LD) holds the tile's rows between the phases, Ts (RPp x
// RPp) a copy of T; csc = per-column output factors 1 / s_B, zi = 1 / s_Z.
template <int RPp>
__device__ void tile_finish(const TcArgs& a, int64_t t, int nseg, int u, int nthr, int bar, float* Ps, float* Ts,
                            const float* csc, float zi, const float* Tn) {
  const int RP = a.RP, RP4 = RP / 4;
  const int64_t o0 = t * BM;
  const int nrow = (int)(a.rows - o0 < BM ? a.rows - o0 : BM);
  __threadfence();   // the other segments' slots: written before their counter increments
  if (u == 0) a.counters[t] = 0u;
  // T (chosen at the kernel's start) is loaded together with the slots: one memory round
  // trip for the whole phase
  constexpr int kTq = kMaxRP * kMaxRP / 4 / 256;   // float4s of T per thread for nthr >= 256
  const int nT4 = Tn ? RP * RP4 : 0;
  float4 tq[kTq];
#pragma unroll
  for (int k = 0; k < kTq; ++k) {
    const int e = u + k * nthr;
    tq[k] = e < nT4 ? __ldg(reinterpret_cast<const float4*>(Tn) + e) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // (1) rows of the tile into Ps: sum of the slots, unscaled.  Consecutive threads take
  // consecutive float4s of a slot (coalesced); four items per thread and up to four slots
  // each are in flight at once.
  const float4* part = reinterpret_cast<const float4*>(a.part + t * a.maxseg * (int64_t)BM * RP);
  const int64_t slot4 = (int64_t)BM * RP4;
  const int nitem = BM * RP4;
  for (int it0 = u; it0 < nitem; it0 += 4 * nthr) {
    float4 acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s0 = 0; s0 < nseg; s0 += 4) {
      float4 v[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int it = it0 + q * nthr;
          v[q][k] = (s0 + k < nseg && it < nitem) ? __ldcg(part + (s0 + k) * slot4 + it) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          acc[q].x += v[q][k].x;
          acc[q].y += v[q][k].y;
          acc[q].z += v[q][k].z;
          acc[q].w += v[q][k].w;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = it0 + q * nthr;
      if (it < nitem) {
        const int row = it / RP4, c = (it % RP4) * 4;
        float* pr = Ps + row * EPI_LD + c;
        const bool live = row < nrow;
        pr[0] = live ? acc[q].x * (csc[c] * zi) : 0.f;
        pr[1] = live ? acc[q].y * (csc[c + 1] * zi) : 0.f;
        pr[2] = live ? acc[q].z * (csc[c + 2] * zi) : 0.f;
        pr[3] = live ? acc[q].w * (csc[c + 3] * zi) : 0.f;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kTq; ++k) {
    const int e = u + k * nthr;
    if (e < nT4) *reinterpret_cast<float4*>(Ts + (e / RP4) * RPp + (e % RP4) * 4) = tq[k];
  }
  named_sync(bar, nthr);
  // (2) Y <- Y T.  A warp takes an 8-column group of the output for one half of the rows
  // (lane: rows lane and lane + 32 of the half), so T is read at warp-uniform addresses;
  // with T upper triangular the group needs rows c <= its last column only.  Results stay
  // in registers until every warp has read Y (at most two items per warp for nthr >= 256).
  if (Tn) {
    const int lane = u & 31, nw = nthr >> 5, CB = RP / 8, nit = 2 * CB;
    float acc[2][2][8];
    int item[2] = {-1, -1};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int itm = (u >> 5) + k * nw;
      if (itm < nit) {
        item[k] = itm;
        const int cg = itm >> 1, r0 = (itm & 1) * 64 + lane, l0 = cg * 8;
        const int cend = a.t_upper ? l0 + 8 : RP;
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[k][i][j] = 0.f;
#pragma unroll 2
        for (int c = 0; c < cend; ++c) {
          const float y0 = Ps[r0 * EPI_LD + c], y1 = Ps[(r0 + 32) * EPI_LD + c];
          const float4 t0 = *reinterpret_cast<const float4*>(Ts + c * RPp + l0);
          const float4 t1 = *reinterpret_cast<const float4*>(Ts + c * RPp + l0 + 4);
          const float tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            acc[k][0][j] = fmaf(y0, tv[j], acc[k][0][j]);
            acc[k][1][j] = fmaf(y1, tv[j], acc[k][1][j]);
          }
        }
      }
    }
    named_sync(bar, nthr);   // every read of Y done before it is overwritten
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (item[k] >= 0) {
        const int cg = item[k] >> 1, r0 = (item[k] & 1) * 64 + lane, l0 = cg * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          Ps[r0 * EPI_LD + l0 + j] = acc[k][0][j];
          Ps[(r0 + 32) * EPI_LD + l0 + j] = acc[k][1][j];
        }
      }
    named_sync(bar, nthr);
  }
  // (3) outputs: rows (float4 per thread), and the split transposed operand (one column
  // l at a time, consecutive threads on consecutive rows)
  if (a.out)
    for (int it = u; it < nrow * RP4; it += nthr) {
      const int row = it / RP4, c = (it % RP4) * 4;
      const float* pr = Ps + row * EPI_LD + c;
      *reinterpret_cast<float4*>(a.out + (o0 + row) * (int64_t)RP + c) = make_float4(pr[0], pr[1], pr[2], pr[3]);
    }
  if (a.bt2)
    for (int it = u; it < RP * BM; it += nthr) {
      const int l = it / BM, row = it % BM;
      if (row < nrow) {
        const float v = Ps[row * EPI_LD + l] * kSkinnyScale;
        const __half c1 = __float2half_rn(v);
        a.bt2[(int64_t)l * a.ldb + o0 + row] = c1;
        a.bt2[(int64_t)(RP + l) * a.ldb + o0 + row] = __float2half_rn((v - __half2float(c1)) * kLoScale);
      }
    }
  // (4) Gram partial Y^T Y of the tile (rows past nrow are zero)
  if (a.gram_mode) {
    const size_t esz = a.gram_mode == 2 ? sizeof(double) : sizeof(float);
    gram_tile(Ps, EPI_LD, RP, a.gram_mode, static_cast<char*>(a.gram_part) + (size_t)t * RP * RP * esz, u, nthr);
  }
  named_sync(bar, nthr);   // Ps and Ts free again
}

// One TMA producer loop over this CTA's stages [g0, g1).  Zsrc stages are two
// 32-column float32 boxes (the second is skipped when it starts at or beyond K);
// skinny-operand stages are one 64-column float16 box.
template <bool IS_A>
__device__ void produce(const CUtensorMap* map, unsigned char* ring, int nslot, size_t slot_bytes, uint32_t box_bytes,
                        uint64_t* fullb, uint64_t* emptyb, int64_t g0, int64_t g1, int64_t ks, int64_t K, Ctl* ctl,
                        volatile int* s_err, int64_t npre = 0) {
  // npre stages were issued already (prefetch_a): continue after them
  int64_t t = (g0 + npre) / ks, kst = (g0 + npre) % ks;
  int s = (int)(npre % nslot);
  uint32_t ph = (uint32_t)((npre / nslot) & 1);
  int64_t issued = npre;
  g0 += npre;
  // Zsrc is streamed once per product and is larger than L2: its lines go first, which
  // leaves L2 to the skinny operand (read by every CTA) and the partial slots
  const uint64_t pol = policy_evict_first();
  for (int64_t g = g0; g < g1 && !*s_err; ++g) {
    if (!mbar_wait(&emptyb[s], ph ^ 1u, kWaitLimit)) { note_timeout(ctl, s_err); break; }
    unsigned char* dst = ring + (size_t)s * slot_bytes;
    if (IS_A) {
      // both boxes always: columns at and past K are zero-filled
      mbar_expect_tx(&fullb[s], 2 * box_bytes);
      tma_load_2d_hint(dst, map, &fullb[s], (int)(kst * BK), (int)(t * BM), pol);
      tma_load_2d_hint(dst + box_bytes, map, &fullb[s], (int)(kst * BK + 32), (int)(t * BM), pol);
    } else {
      mbar_expect_tx(&fullb[s], box_bytes);
      tma_load_2d(dst, map, &fullb[s], (int)(kst * BK), 0);
    }
    ++issued;
    if (++kst == ks) { kst = 0; ++t; }
    if (++s == nslot) { s = 0; ph ^= 1u; }
  }
  // Every copy issued has landed before the CTA may exit (immediate in the normal case).
  for (int64_t j = (issued > nslot ? issued - nslot : 0); j < issued; ++j)
    if (!mbar_wait(&fullb[(int)(j % nslot)], (uint32_t)((j / nslot) & 1), kWaitLimit)) note_timeout(ctl, s_err);
}

// The first stages of this CTA's Zsrc range into the empty ring (every slot is free at the
// start), issued before the programmatic wait on the preceding kernel when that kernel
// leaves Zsrc unchanged: the stream then starts as soon as the skinny operand lands.
// Returns the number of stages issued; produce() continues after them and drains them on
// an abort like its own.
__device__ int64_t prefetch_a(const CUtensorMap* map, unsigned char* ring, uint64_t* fullb, int64_t g0, int64_t g1,
                              int64_t ks) {
  const uint64_t pol = policy_evict_first();
  const int64_t n = (g1 - g0 < NA) ? g1 - g0 : NA;
  int64_t t = g0 / ks, kst = g0 % ks;
  for (int64_t s = 0; s < n; ++s) {
    unsigned char* dst = ring + (size_t)s * kStageA;
    mbar_expect_tx(&fullb[s], 2 * (uint32_t)kBoxA);
    tma_load_2d_hint(dst, map, &fullb[s], (int)(kst * BK), (int)(t * BM), pol);
    tma_load_2d_hint(dst + kBoxA, map, &fullb[s], (int)(kst * BK + 32), (int)(t * BM), pol);
    if (++kst == ks) { kst = 0; ++t; }
  }
  return n > 0 ? n : 0;
}

// Warp-uniform bounded wait: lane 0 polls, the warp follows (__syncwarp orders the
// other lanes' later accesses after lane 0's acquire).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, kWaitLimit) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

template <int RPp, bool PRESCALED>
__global__ void __launch_bounds__(kThreads, 1)
k_prod_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  Ctl* ctl = a.ctl;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm + kOffA;
  unsigned char* sB = sm + kOffB;
  float* Ps = reinterpret_cast<float*>(sm + kOffA);   // completion staging: the ring, once idle
  float* Ts = Ps + BM * EPI_LD;
  __shared__ uint64_t afull[NA], aempty[NA], bfull[NS], tfull[NS], sfree[NS], cpdone[NS];
  __shared__ uint64_t accfull[2], accempty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_err;   // set by any role that gives up; every loop polls it
  __shared__ int s_stop, s_last;   // epilogue-wide decisions, written between two named barriers
  __shared__ int s_npend;   // tiles this CTA completes (listed in a.pend), done at its end
  __shared__ float s_csc[kMaxRP];
  __shared__ float s_zi;
  __shared__ const float* s_tn;   // the normaliser of this launch (by slot parity)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x;
  const int64_t S = a.S, ks = a.ks, K = a.K;
  const int G = a.G;
  const int64_t g0 = (int64_t)c * S / G, g1 = (int64_t)(c + 1) * S / G;
  int64_t npre = 0;   // Zsrc stages issued before the programmatic wait (thread 0, the producer)
  if (tid == 0) {
    for (int s = 0; s < NA; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);   // the copier's commit
    }
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&tfull[s], kConvWarps);
      mbar_init(&sfree[s], 1);
      mbar_init(&cpdone[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 4);
    }
    mbar_init(&mma_done, 1);
    fence_barrier_init();
    if (a.z_prefetch) npre = prefetch_a(&mapA, sA, afull, g0, g1, ks);
  }
  if (warp == 1) tmem_alloc(&tmem_base, kTmemCols);
  // Launched as a programmatic dependent of the previous product: everything above ran
  // while that product completed its tiles; apart from the prefetch of Zsrc (which the
  // preceding kernels do not write), no global memory is touched before this.
  pdl_wait();
  if (tid == 0) {
    // Iteration already abandoned, or Z outgrew its scale in the last S-step (the caller
    // rescales it): do nothing, and make the rest of the iteration skip too.
    s_err = (ctl && (ctl->abort || ctl->range_err)) ? 2 : 0;
    if (ctl && ctl->range_err) ctl->abort = 1;
    s_npend = 0;
    s_zi = a.zscale ? a.zscale[1] : 1.f;
    s_tn = (ctl && ctl->slot_parity) ? a.Tn1 : a.Tn0;
  }
  if (tid < kMaxRP) s_csc[tid] = (tid < a.RP && a.cscale) ? a.cscale[tid] : 1.f;
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer: Zsrc tiles ----------------
    if (lane == 0)
      produce<true>(&mapA, sA, NA, kStageA, (uint32_t)kBoxA, afull, aempty, g0, g1, ks, K, ctl, &s_err, npre);
  } else if (warp == 14) {
    // ---------------- TMA producer: skinny-operand tiles ----------------
    if (lane == 0)
      produce<false>(&mapB, sB, NS, kStageB, (uint32_t)(2 * a.RP * BK * 2), bfull, sfree, g0, g1, ks, K, ctl,
                     &s_err);
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const int RP = a.RP;
      const uint32_t id_hi = idesc_f16(BM, 2 * RP), id_lo = idesc_f16(BM, RPp);   // RPp: RP rounded up to 16
      int ch = 0;   // chunks issued by this CTA
      int st = 0;
      uint32_t ph = 0;
      int64_t kst = g0 % ks;
      int64_t g = g0;
      while (g < g1 && !s_err) {
        // this chunk: up to kChunk stages, not past the end of the tile or of the range
        int64_t n = ks - kst;
        if (n > kChunk) n = kChunk;
        if (n > g1 - g) n = g1 - g;
        const int b = ch & 1;
        if (!mbar_wait(&accempty[b], (uint32_t)(((ch >> 1) & 1) ^ 1), kWaitLimit)) { note_timeout(ctl, &s_err); break; }
        tc_fence_after();
        const uint32_t dcol = tbase + (uint32_t)(b * 128);
        uint32_t acc = 0;
        for (int64_t e = 0; e < n; ++e) {
          if (!mbar_wait(&tfull[st], ph, kWaitLimit)) { note_timeout(ctl, &s_err); break; }
          tc_fence_after();
          const uint64_t db = sdesc_k128(sB + (size_t)st * kStageB);
          // slot columns: [h of K 0..31 | l of K 0..31 | h of K 32..63 | l of K 32..63], 16 each
          const uint32_t aslot = tbase + kTA0 + (uint32_t)st * kTASlot;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t off = (uint64_t)((kk * 16 * 2) >> 4);   // 32 bytes per 16-wide K step
            const uint32_t ah = aslot + (uint32_t)((kk >> 1) * 32 + (kk & 1) * 8);
            mma_f16_ta(dcol, ah, db + off, id_hi, acc);
            mma_f16_ta(dcol + RP, ah + 16, db + off, id_lo, 1u);
            acc = 1u;
          }
          mma_commit(&sfree[st]);
          if (++st == NS) { st = 0; ph ^= 1u; }
        }
        if (s_err) break;
        mma_commit(&accfull[b]);
        ++ch;
        g += n;
        kst += n;
        if (kst == ks) kst = 0;
      }
      mma_commit(&mma_done);
      if (!mbar_wait(&mma_done, 0, kWaitLimit)) note_timeout(ctl, &s_err);
    }
  } else if (warp == 15) {
    // ---------------- copier: landed Zsrc stage -> its TMEM stage slot ----------------
    if (lane == 0) {
      int sa = 0, st = 0;
      uint32_t pha = 0, ph = 0;
      int64_t n = 0;
      for (int64_t g = g0; g < g1 && !s_err; ++g) {
        if (!mbar_wait(&afull[sa], pha, kWaitLimit) || !mbar_wait(&sfree[st], ph ^ 1u, kWaitLimit)) {
          note_timeout(ctl, &s_err);
          break;
        }
        tc_fence_after();
        const uint32_t dst = tbase + kTA0 + (uint32_t)st * kTASlot;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const uint64_t d = sdesc_k128(sA + (size_t)sa * kStageA + b * kBoxA);
#pragma unroll
          for (int k = 0; k < 4; ++k) tmem_cp_128x256b(dst + (uint32_t)(b * 32 + k * 8), d + (uint64_t)(2 * k));
        }
        mma_commit(&cpdone[st]);   // the converters may read the slot
        mma_commit(&aempty[sa]);   // the shared-memory slot may be refilled
        ++n;
        if (++sa == NA) { sa = 0; pha ^= 1u; }
        if (++st == NS) { st = 0; ph ^= 1u; }
      }
      // the last copies have finished reading shared memory and writing TMEM
      for (int64_t j = (n > NS ? n - NS : 0); j < n; ++j)
        if (!mbar_wait(&cpdone[(int)(j % NS)], (uint32_t)((j / NS) & 1), kWaitLimit)) note_timeout(ctl, &s_err);
    }
  } else if (warp < 2 + kConvWarps) {
    // ---------------- converters: float32 stage in TMEM -> packed (h1, h2) in place ----------------
    const int q = (warp - 2) >> 2;              // 32-column half of the tile handled by this warp
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;   // this warp's TMEM lane quarter
    const float zs = (!PRESCALED && a.zscale) ? a.zscale[0] : 1.f;
    int st = 0;
    uint32_t ph = 0;
    for (int64_t g = g0; g < g1; ++g) {
      if (__any_sync(0xffffffffu, s_err != 0)) break;
      if (!warp_wait(&cpdone[st], ph, lane)) {
        if (lane == 0) note_timeout(ctl, &s_err);
        break;
      }
      tc_fence_after();
      const uint32_t ta = tbase + kTA0 + (uint32_t)st * kTASlot + tlane + (uint32_t)(q * 32);
      float xs[32];
      tmem_ld32(ta, xs);
      uint32_t h[16], l2[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float x0 = xs[2 * k], x1 = xs[2 * k + 1];
        if (!PRESCALED) {
          x0 *= zs;
          x1 *= zs;
        }
        const float h0 = __uint_as_float(__float_as_uint(x0) & 0xFFFFE000u);
        const float h1 = __uint_as_float(__float_as_uint(x1) & 0xFFFFE000u);
        h[k] = pack_h2(h0, h1);
        l2[k] = pack_h2((x0 - h0) * kLoScale, (x1 - h1) * kLoScale);
      }
      tmem_st16(ta, h);
      tmem_st16(ta + 16, l2);
      tmem_wait_st();
      tc_fence_before();
      // the skinny tile of this stage has landed too: the MMA issuer waits on tfull alone
      if (!warp_wait(&bfull[st], ph, lane)) {
        if (lane == 0) note_timeout(ctl, &s_err);
        break;
      }
      if (lane == 0) mbar_arrive(&tfull[st]);
      if (++st == NS) { st = 0; ph ^= 1u; }
    }
  } else {
    // ---------------- epilogue: TMEM -> running sums -> partial slot, tile completion ----------------
    // The four warps take every decision together (flag written between two named
    // barriers), so no warp can leave while the others wait at a barrier.
    const int et = tid - 32 * (2 + kConvWarps);
    const int q4 = warp & 3;                 // TMEM lane quarter this warp may access
    const int row = q4 * 32 + lane;          // tile row held by this thread
    const uint32_t tlane = (uint32_t)(q4 * 32) << 16;
    int ch = 0, npend = 0;
    int64_t g = g0;
    for (;;) {
      named_sync(1, BM);
      if (et == 0) s_stop = (g >= g1) || s_err;
      named_sync(1, BM);
      if (s_stop) break;
      const int64_t t = g / ks;
      const int64_t tend = ((t + 1) * ks < g1) ? (t + 1) * ks : g1;
      float y[RPp];
#pragma unroll
      for (int l = 0; l < RPp; ++l) y[l] = 0.f;
      bool failed = false;
      for (; g < tend; g = (g + kChunk < tend) ? g + kChunk : tend, ++ch) {
        if (failed) continue;                // keep the loop count; nothing more to read
        const int b = ch & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&accfull[b], (uint32_t)((ch >> 1) & 1), kWaitLimit))) {
          if (lane == 0) note_timeout(ctl, &s_err);
          failed = true;
          continue;
        }
        tc_fence_after();
        const uint32_t taddr = tbase + (uint32_t)(b * 128) + tlane;
#pragma unroll
        for (int c0 = 0; c0 < RPp; c0 += 8) {
          if (c0 < a.RP) {
            float vh[8], vl[8];
            tmem_ld8(taddr + c0, vh);
            tmem_ld8(taddr + a.RP + c0, vl);
#pragma unroll
            for (int l = 0; l < 8; ++l) y[c0 + l] += fmaf(vl[l], kLoInv, vh[l]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty[b]);
      }
      named_sync(1, BM);
      if (et == 0) s_stop = s_err;
      named_sync(1, BM);
      if (s_stop) break;
      const int64_t c_first = cta_of(t * ks, S, G);
      const int nseg = (int)(cta_of((t + 1) * ks - 1, S, G) - c_first + 1);
      const int slot = (int)(c - c_first);
      float* p = a.part + ((t * a.maxseg + slot) * BM + row) * (int64_t)a.RP;
#pragma unroll
      for (int l = 0; l < RPp; l += 4)
        if (l < a.RP) *reinterpret_cast<float4*>(p + l) = make_float4(y[l], y[l + 1], y[l + 2], y[l + 3]);
      __threadfence();
      named_sync(1, BM);
      if (et == 0) s_last = (atomicAdd(&a.counters[t], 1u) == (unsigned)(nseg - 1));
      named_sync(1, BM);
      if (s_last) {
        if (et == 0) {
          if (npend < a.maxpend) a.pend[(int64_t)c * a.maxpend + npend] = (int)t;
          else if (ctl) ctl->abort = 1;   // cannot happen with the host's bound; never skip silently
        }
        ++npend;
      }
    }
    if (et == 0) s_npend = npend;
  }

  tc_fence_before();
  __syncthreads();
  pdl_launch_dependents();   // the stream is done: the next product may start its prologue
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, kTmemCols);
  }
  // completions: the whole CTA on each tile whose last segment was this CTA's
  const int np = s_err ? 0 : (s_npend < a.maxpend ? s_npend : a.maxpend);
  for (int k = 0; k < np; ++k) {
    const int64_t t = a.pend[(int64_t)c * a.maxpend + k];
    const int64_t c_first = cta_of(t * ks, S, G);
    const int nseg = (int)(cta_of((t + 1) * ks - 1, S, G) - c_first + 1);
    tile_finish<RPp>(a, t, nseg, tid, kThreads, 0, Ps, Ts, s_csc, s_zi, s_tn);
  }
}

// ---- 16-bit streaming product (precision form) -------------------------------------------
// part/out = Z16 (rows x K, float16 copy of (X - S) s_Z, rounded) * B with B in its two-term
// split c1 + 2^-11 c2 (rows 0..2RP-1 of bt2): one float16 MMA of N = 2 RP per stage gives
// Z16 c1 and Z16 c2 side by side in tensor memory, summed as hi + 2^-11 lo in the
// epilogue, float32 accumulation.  Z16 carries about 2^-12 relative rounding per element
// (fixed for the whole chain); B is exact to about 2^-22, so the chain's error is that of
// X's rounding alone (rounding B to one float16 term as well adds a fresh 2^-12 per
// product, which the float32 correction pass can no longer remove when sigma_r and
// sigma_{r+1} are close).  The Z16 tile of a stage is one 128-row x 64-column box that
// the MMA reads straight from shared memory (no conversion), so the stream moves half
// the bytes of the float32 kernel.  Same stream-K split, partial slots and deferred tile
// completion as k_prod_tc.  RP <= 32 (the precision form's bound on r).
// Warps: 0 TMA producer of Z16 tiles, 1 MMA issuer (TMEM owner), 2-5 epilogue, 6 TMA
// producer of the skinny operand, 7 spare (completion only).
constexpr int NA16 = 10, NS16 = 6, kThreads16 = 256;
constexpr size_t kStageA16 = (size_t)BM * 128;                 // 64 halves x 128 rows = 16 KB
constexpr int kMaxRP16 = 32;                                   // RP bound of the 16-bit kernel
constexpr size_t kStageB16 = (size_t)2 * kMaxRP16 * 128;       // up to 2 x 32 rows of 64 halves = 8 KB
constexpr size_t kOffB16 = NA16 * kStageA16;
constexpr size_t kTc16Smem = kOffB16 + NS16 * kStageB16 + 1024;
static_assert(kEpiBytes <= NA16 * kStageA16, "completion staging fits the 16-bit ring");
static_assert(kTc16Smem <= 232448 - 1024, "shared memory of the 16-bit product");

template <int RPp>
__global__ void __launch_bounds__(kThreads16, 1)
k_prod_h16(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  Ctl* ctl = a.ctl;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = sm;
  unsigned char* sB = sm + kOffB16;
  float* Ps = reinterpret_cast<float*>(sm);   // completion staging: the ring, once idle
  float* Ts = Ps + BM * EPI_LD;
  __shared__ uint64_t afull[NA16], aempty[NA16], bfull[NS16], bempty[NS16];
  __shared__ uint64_t accfull[2], accempty[2], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_err;
  __shared__ int s_stop, s_last, s_npend;
  __shared__ float s_csc[kMaxRP];
  __shared__ float s_zi;
  __shared__ const float* s_tn;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x;
  const int64_t S = a.S, ks = a.ks;
  const int G = a.G;
  const int64_t g0 = (int64_t)c * S / G, g1 = (int64_t)(c + 1) * S / G;
  static_assert(RPp <= kMaxRP16, "16-bit kernel: RP <= 32");
  const uint32_t bbytes = (uint32_t)(2 * a.RP * 128);   // c1 and c2 rows of the stage
  if (tid == 0) {
    for (int s = 0; s < NA16; ++s) {
      mbar_init(&afull[s], 1);
      mbar_init(&aempty[s], 1);
    }
    for (int s = 0; s < NS16; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 4);
    }
    mbar_init(&mma_done, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, 128);
  pdl_wait();   // see k_prod_tc
  if (tid == 0) {
    s_err = (ctl && (ctl->abort || ctl->range_err)) ? 2 : 0;
    if (ctl && ctl->range_err) ctl->abort = 1;
    s_npend = 0;
    s_zi = a.zscale ? a.zscale[1] : 1.f;
    s_tn = (ctl && ctl->slot_parity) ? a.Tn1 : a.Tn0;
  }
  if (tid < kMaxRP) s_csc[tid] = (tid < a.RP && a.cscale) ? a.cscale[tid] : 1.f;
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0 || warp == 6) {
    // ---------------- TMA producers: Z16 tiles (warp 0), skinny-operand tiles (warp 6) ----------
    if (lane == 0) {
      const bool isA = warp == 0;
      const int nslot = isA ? NA16 : NS16;
      uint64_t* fullb = isA ? afull : bfull;
      uint64_t* emptyb = isA ? aempty : bempty;
      int64_t t = g0 / ks, kst = g0 % ks, issued = 0;
      int s = 0;
      uint32_t ph = 0;
      const uint64_t pol = policy_evict_first();   // Z16 streamed once per product
      for (int64_t g = g0; g < g1 && !s_err; ++g) {
        if (!mbar_wait(&emptyb[s], ph ^ 1u, kWaitLimit)) { note_timeout(ctl, &s_err); break; }
        if (isA) {
          mbar_expect_tx(&fullb[s], (uint32_t)kStageA16);
          tma_load_2d_hint(sA + (size_t)s * kStageA16, &mapA, &fullb[s], (int)(kst * BK), (int)(t * BM), pol);
        } else {
          mbar_expect_tx(&fullb[s], bbytes);
          tma_load_2d(sB + (size_t)s * kStageB16, &mapB, &fullb[s], (int)(kst * BK), 0);
        }
        ++issued;
        if (++kst == ks) { kst = 0; ++t; }
        if (++s == nslot) { s = 0; ph ^= 1u; }
      }
      for (int64_t j = (issued > nslot ? issued - nslot : 0); j < issued; ++j)
        if (!mbar_wait(&fullb[(int)(j % nslot)], (uint32_t)((j / nslot) & 1), kWaitLimit)) note_timeout(ctl, &s_err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id = idesc_f16(BM, 2 * a.RP);   // [Z16 c1 | Z16 c2], RP multiple of 8
      int ch = 0, sa = 0, sb = 0;
      uint32_t pha = 0, phb = 0;
      int64_t kst = g0 % ks, g = g0;
      while (g < g1 && !s_err) {
        int64_t n = ks - kst;
        if (n > kChunk) n = kChunk;
        if (n > g1 - g) n = g1 - g;
        const int b = ch & 1;
        if (!mbar_wait(&accempty[b], (uint32_t)(((ch >> 1) & 1) ^ 1), kWaitLimit)) { note_timeout(ctl, &s_err); break; }
        tc_fence_after();
        const uint32_t dcol = tbase + (uint32_t)(b * 64);
        uint32_t acc = 0;
        for (int64_t e = 0; e < n; ++e) {
          if (!mbar_wait(&afull[sa], pha, kWaitLimit) || !mbar_wait(&bfull[sb], phb, kWaitLimit)) {
            note_timeout(ctl, &s_err);
            break;
          }
          tc_fence_after();
          const uint64_t da = sdesc_k128(sA + (size_t)sa * kStageA16), db = sdesc_k128(sB + (size_t)sb * kStageB16);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t off = (uint64_t)((kk * 16 * 2) >> 4);   // 32 bytes per 16-wide K step
            mma_bf16(dcol, da + off, db + off, id, acc);
            acc = 1u;
          }
          mma_commit(&aempty[sa]);
          mma_commit(&bempty[sb]);
          if (++sa == NA16) { sa = 0; pha ^= 1u; }
          if (++sb == NS16) { sb = 0; phb ^= 1u; }
        }
        if (s_err) break;
        mma_commit(&accfull[b]);
        ++ch;
        g += n;
        kst += n;
        if (kst == ks) kst = 0;
      }
      mma_commit(&mma_done);
      if (!mbar_wait(&mma_done, 0, kWaitLimit)) note_timeout(ctl, &s_err);
    }
  } else if (warp >= 2 && warp < 6) {
    // ---------------- epilogue: TMEM -> running sums -> partial slot ----------------
    const int et = tid - 64;
    const int q4 = warp & 3;
    const int row = q4 * 32 + lane;
    const uint32_t tlane = (uint32_t)(q4 * 32) << 16;
    int ch = 0, npend = 0;
    int64_t g = g0;
    for (;;) {
      named_sync(1, BM);
      if (et == 0) s_stop = (g >= g1) || s_err;
      named_sync(1, BM);
      if (s_stop) break;
      const int64_t t = g / ks;
      const int64_t tend = ((t + 1) * ks < g1) ? (t + 1) * ks : g1;
      float y[RPp];
#pragma unroll
      for (int l = 0; l < RPp; ++l) y[l] = 0.f;
      bool failed = false;
      for (; g < tend; g = (g + kChunk < tend) ? g + kChunk : tend, ++ch) {
        if (failed) continue;
        const int b = ch & 1;
        if (!__all_sync(0xffffffffu, mbar_wait(&accfull[b], (uint32_t)((ch >> 1) & 1), kWaitLimit))) {
          if (lane == 0) note_timeout(ctl, &s_err);
          failed = true;
          continue;
        }
        tc_fence_after();
        const uint32_t taddr = tbase + (uint32_t)(b * 64) + tlane;
#pragma unroll
        for (int c0 = 0; c0 < RPp; c0 += 8) {
          if (c0 < a.RP) {
            float vh[8], vl[8];
            tmem_ld8(taddr + c0, vh);
            tmem_ld8(taddr + a.RP + c0, vl);
#pragma unroll
            for (int l = 0; l < 8; ++l) y[c0 + l] += fmaf(vl[l], kLoInv, vh[l]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accempty[b]);
      }
      named_sync(1, BM);
      if (et == 0) s_stop = s_err;
      named_sync(1, BM);
      if (s_stop) break;
      const int64_t c_first = cta_of(t * ks, S, G);
      const int nseg = (int)(cta_of((t + 1) * ks - 1, S, G) - c_first + 1);
      const int slot = (int)(c - c_first);
      float* p = a.part + ((t * a.maxseg + slot) * BM + row) * (int64_t)a.RP;
#pragma unroll
      for (int l = 0; l < RPp; l += 4)
        if (l < a.RP) *reinterpret_cast<float4*>(p + l) = make_float4(y[l], y[l + 1], y[l + 2], y[l + 3]);
      __threadfence();
      named_sync(1, BM);
      if (et == 0) s_last = (atomicAdd(&a.counters[t], 1u) == (unsigned)(nseg - 1));
      named_sync(1, BM);
      if (s_last) {
        if (et == 0) {
          if (npend < a.maxpend) a.pend[(int64_t)c * a.maxpend + npend] = (int)t;
          else if (ctl) ctl->abort = 1;
        }
        ++npend;
      }
    }
    if (et == 0) s_npend = npend;
  }

  tc_fence_before();
  __syncthreads();
  pdl_launch_dependents();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 128);
  }
  const int np = s_err ? 0 : (s_npend < a.maxpend ? s_npend : a.maxpend);
  for (int k = 0; k < np; ++k) {
    const int64_t t = a.pend[(int64_t)c * a.maxpend + k];
    const int64_t c_first = cta_of(t * ks, S, G);
    const int nseg = (int)(cta_of((t + 1) * ks - 1, S, G) - c_first + 1);
    tile_finish<RPp>(a, t, nseg, tid, kThreads16, 0, Ps, Ts, s_csc, s_zi, s_tn);
  }
}

// Column c of a row-major rows x RP operand B -> rows c and RP + c of the split
// transposed float16 operand, scaled by the power of two 2^e_c that brings the column's
// largest magnitude into [2^9, 2^10); cscale[c] = 2^-e_c undoes it.  One block per column.
__global__ void k_split_t(const float* __restrict__ B, int64_t rows, int RP, __half* __restrict__ bt2, int64_t ldb,
                          float* __restrict__ cscale, const int* skip) {
  if (block_skip(skip)) return;
  const int col = blockIdx.x;
  __shared__ float red[32];
  __shared__ float s_scale;
  float m = 0.f;
  if (col < RP)
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) m = fmaxf(m, fabsf(B[i * RP + col]));
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
    int e = 0;
    if (mm > 0.f && isfinite(mm)) {
      int ex;
      frexpf(mm, &ex);   // mm in [2^(ex-1), 2^ex)
      e = 10 - ex;
      e = e < -120 ? -120 : (e > 120 ? 120 : e);
    }
    s_scale = ldexpf(1.f, e);
    if (col < RP) cscale[col] = ldexpf(1.f, -e);
  }
  __syncthreads();
  const float sc = s_scale;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    const float v = (col < RP) ? B[i * RP + col] * sc : 0.f;
    const __half c1 = __float2half_rn(v);
    bt2[(int64_t)col * ldb + i] = c1;
    bt2[(int64_t)(RP + col) * ldb + i] = __float2half_rn((v - __half2float(c1)) * kLoScale);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

// A tensor map over a row-major matrix (rows x cols, row stride ld elements) read in
// boxes of 128 bytes of columns (32 float32 or 64 float16) x box_rows rows with the
// 128-byte swizzle.
static bool make_tmap(void* map, CUtensorMapDataType dt, int esize, const void* base, int64_t rows, int64_t cols,
                      int64_t ld, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esize), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(reinterpret_cast<CUtensorMap*>(map), dt, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
bool make_tmap_f32(void* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  return make_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, rows, cols, ld, box_rows);
}
bool make_tmap_f16(void* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  return make_tmap(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, rows, cols, ld, box_rows);
}

int tc_rpp(int RP) { return (RP + 15) / 16 * 16; }

void launch_split_t(const float* B, int64_t rows, int RP, void* bt2, int64_t ldb, float* cscale, cudaStream_t st,
                    const int* skip) {
  k_split_t<<<RP, 256, 0, st>>>(B, rows, RP, reinterpret_cast<__half*>(bt2), ldb, cscale, skip);
}

TcGeom tc_geometry(int64_t rows, int64_t K, int nsm) {
  TcGeom g;
  g.tiles = (rows + BM - 1) / BM;
  g.ks = (K + BK - 1) / BK;
  g.S = g.tiles * g.ks;
  // Leave a few SMs without a product CTA: the r x r kernels of the side stream run
  // there instead of holding an SM that a persistent CTA (which needs the whole shared
  // memory) would otherwise wait for.
  const int ncta = nsm > 16 ? nsm - 4 : nsm;
  g.G = (int)(g.S < ncta ? g.S : ncta);
  int maxseg = 1;
  for (int64_t t = 0; t < g.tiles; ++t) {
    const int64_t cf = ((t * g.ks + 1) * g.G - 1) / g.S;
    const int64_t cl = (((t + 1) * g.ks) * g.G - 1) / g.S;
    if (cl - cf + 1 > maxseg) maxseg = (int)(cl - cf + 1);
  }
  g.maxseg = maxseg;
  // tiles meeting one CTA's range (its completions are listed for the end of the kernel)
  const int64_t span = (g.S + g.G - 1) / g.G;
  g.maxpend = (int)((span + g.ks - 1) / g.ks + 1);
  return g;
}

template <int RPp, bool PS>
static cudaError_t prep_one() {
  return cudaFuncSetAttribute(k_prod_tc<RPp, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
}

template <int RPp>
static cudaError_t prep16() {
  return cudaFuncSetAttribute(k_prod_h16<RPp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTc16Smem);
}

cudaError_t prepare_tc_kernels() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = prep16<16>();
  if (e == cudaSuccess) e = prep16<32>();
  if (e == cudaSuccess) e = prep_one<16, false>();
  if (e == cudaSuccess) e = prep_one<32, false>();
  if (e == cudaSuccess) e = prep_one<48, false>();
  if (e == cudaSuccess) e = prep_one<64, false>();
  if (e == cudaSuccess) e = prep_one<16, true>();
  if (e == cudaSuccess) e = prep_one<32, true>();
  if (e == cudaSuccess) e = prep_one<48, true>();
  if (e == cudaSuccess) e = prep_one<64, true>();
  return e;
}

// Launch with the programmatic-stream-serialization attribute when pdl is set: the kernel
// may begin (barrier set-up, tensor-memory allocation) while the preceding kernel of the
// stream finishes, and waits for it in pdl_wait() before its first global access.
template <typename Kern>
static void launch_tc(Kern kern, unsigned grid, unsigned block, size_t smem, cudaStream_t st, bool pdl,
                      const CUtensorMap& A, const CUtensorMap& B, const TcArgs& a) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, A, B, a);
}

void launch_prod_tc(const TcLaunch& l, cudaStream_t st) {
  TcArgs a;
  a.rows = l.rows;
  a.K = l.K;
  a.RP = l.RP;
  a.ks = l.geom.ks;
  a.S = l.geom.S;
  a.G = l.geom.G;
  a.maxseg = l.geom.maxseg;
  a.part = l.part;
  a.counters = l.counters;
  a.out = l.out;
  a.bt2 = reinterpret_cast<__half*>(l.bt2);
  a.ldb = l.ldb;
  a.Tn0 = l.Tn[0];
  a.Tn1 = l.Tn[1];
  a.cscale = l.cscale;
  a.zscale = l.zscale;
  a.gram_part = l.gram_part;
  a.gram_mode = l.gram_mode;
  a.z_prefetch = l.z_prefetch;
  a.t_upper = l.t_upper;
  a.pend = l.pend;
  a.maxpend = l.geom.maxpend;
  a.ctl = l.ctl;
  const CUtensorMap& A = *reinterpret_cast<const CUtensorMap*>(l.mapA);
  const CUtensorMap& B = *reinterpret_cast<const CUtensorMap*>(l.mapB);
  a.prescaled = l.prescaled;
  const int rpp = tc_rpp(l.RP);
  const bool pdl = l.pdl != 0;
  const unsigned G = (unsigned)a.G;
  if (l.half_a) {
    switch (rpp) {
      case 16: launch_tc(k_prod_h16<16>, G, kThreads16, kTc16Smem, st, pdl, A, B, a); break;
      case 32: launch_tc(k_prod_h16<32>, G, kThreads16, kTc16Smem, st, pdl, A, B, a); break;
      default: if (l.ctl) cudaMemsetAsync(&l.ctl->abort, 0xff, sizeof(int), st); break;   // RP > 32: rejected at init
    }
  } else if (l.prescaled) {
    switch (rpp) {
      case 16: launch_tc(k_prod_tc<16, true>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
      case 32: launch_tc(k_prod_tc<32, true>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
      case 48: launch_tc(k_prod_tc<48, true>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
      default: launch_tc(k_prod_tc<64, true>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
    }
  } else {
    switch (rpp) {
      case 16: launch_tc(k_prod_tc<16, false>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
      case 32: launch_tc(k_prod_tc<32, false>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
      case 48: launch_tc(k_prod_tc<48, false>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
      default: launch_tc(k_prod_tc<64, false>, G, kThreads, kTcSmem, st, pdl, A, B, a); break;
    }
  }
}

}  // namespace godec
