// Host side of the C ABI declared in include/godec.h: context and workspace,
// the launch sequence of one iteration of Algorithm 1 (captured into CUDA
// graphs and replayed), recovery from aborted iterations (rank drop,
// candidate overflow, ill-conditioned lagged normalisers), and the getters.
//
// Power chain of one L-step (products i = 0 .. 6q+2, alternating Z and Z^T):
//  * exact path: every product is orthonormalised by CholeskyQR on the
//    critical path;
//  * fast path (from the second iteration on): product i is normalised in its
//    own epilogue by T_i, the inverse of the factor that orthonormalised slot i
//    in the previous iteration; the Cholesky factor of the result is computed
//    on a side stream and becomes next iteration's T_i.  Only Q2 and Q1 (the
//    bases L is built on) get an exact CholeskyQR2 on the critical path.
// In both paths the core of eq. (mlr_app) is M = R_fin * (factors applied in the
// last chain), exact by construction.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "godec_internal.cuh"

using namespace godec;

namespace {
constexpr int kEvents = 160;
constexpr int kRefineParts = 1024;   // row partitions of the correction's cross Grams (128 rows each)
constexpr int kMaxBackoff = 32;       // longest run of exact iterations after repeated alarms
constexpr float kAlarmRatio = 30.f;   // lagged normaliser: max/min Cholesky diagonal of Q~
// Fast path, Q2 and Q1: one CholeskyQR pass on the lagged-normalised product; a
// diagonal spread of its factor above this ratio (condition number of the product)
// sends the iteration to the exact path instead of a second pass.
constexpr float kCqr1Ratio = 1.5f;
constexpr int kNaiveColdSteps = 6;    // naive GoDec: power steps on X before the first L-step
}

struct godec_ctx {
  godec_params p;
  int r = 0;          // current rank (drops after a failed rank test)
  int RP = 0;         // padded width of the skinny buffers (from the initial r)
  int nprod = 0;      // 6q + 3
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;    // private stream used while capturing
  cudaStream_t side_st = nullptr;   // off-critical-path work of the power chain
  cudaStream_t rank_st = nullptr;   // the rank test, joined before the S-step commits
  bool rank_forked = false;
  cudaEvent_t ev[kEvents] = {};
  int ev_used = 0;
  int dev = 0, nsm = 0;   // nsm: the SMs this problem's grids are sized for (its budget)
  int nsm_dev = 0;          // SMs of the device
  size_t npart_cap = 0, npend_cap = 0;   // stream-K buffers (sized for the whole device)
  const float* X = nullptr;
  float* Z = nullptr;                  // m x ldz   working X - S
  int64_t ldz = 0;
  float* Zt = nullptr;                 // n x ldzt  its transpose
  int64_t ldzt = 0;
  void* Z16 = nullptr;
  void* Zt16 = nullptr;
  float* A1 = nullptr;                 // n x RP; columns >= r kept at zero
  float* A1_orig = nullptr;            // n x RP as given (restored by godec_reset)
  float* P = nullptr;                  // max(m,n) x RP
  float* Q1 = nullptr;                 // m x RP
  float* Q2 = nullptr;                 // n x RP
  float* U = nullptr;                  // m x RP
  float* V = nullptr;                  // n x RP
  float* sigma = nullptr;              // RP
  float* Um = nullptr;
  float* Vm = nullptr;
  // Operands of the tensor-core products in float16 split transposed form, each
  // 2 RP x ldb halves.  bt2[0] is written by even products (read by odd ones, K = m),
  // bt2[1] by odd products (read by even ones, K = n), bt2[2] holds A1 (read by product 0).
  void* bt2 = nullptr;
  int64_t ldb = 0;
  int RPp = 0;
  float* cs = nullptr;                 // [2][RP] output factors: A1's column scales, 1 / kSkinnyScale
  float* rescale_tmp = nullptr;        // 2 floats: factor applied by rescale_z
  // tensor maps: 0 Z, 1 Z^T, 2-4 bt2[0..2], 5 X, 6-7 Lsplit A, B; precision form: 8 Z16,
  // 9 Z16^T, 13-14 bt2[3] over K = n and K = m (10-12 unused)
  alignas(64) unsigned char tmap[16][128];
  // precision form: float32 correction scratch
  float *RA = nullptr, *RB = nullptr, *Wa = nullptr, *Wb = nullptr, *Qa = nullptr, *Qb = nullptr, *Qtmp = nullptr;
  float *Rf = nullptr, *cs_ref = nullptr;
  double *rf_part = nullptr, *rf_g = nullptr, *rf_C = nullptr, *rf_core = nullptr, *rf_U = nullptr, *rf_V = nullptr;
  void* LA = nullptr;                  // m x 128 halves: float16 split of U diag(sqrt(sigma s_Z))
  void* LB = nullptr;                  // n x 128 halves: float16 split of V diag(sqrt(sigma s_Z))
  TcGeom tg[2];                        // work split of even (Z) and odd (Z^T) products
  float* part = nullptr;               // stream-K partial slots
  unsigned* counters = nullptr;        // per-tile arrival counters
  int* pend = nullptr;                 // per-CTA lists of deferred tile completions
  int64_t ncounters = 0;
  char* gparts = nullptr;              // per product: tiles x RP x RP Gram partials (double room)
  size_t gpart_stride = 0;
  double* g64 = nullptr;               // per product reduced Gram, + 2 for the CholeskyQR2 rounds
  float* g32 = nullptr;                // the same in float (read by the float32 factorisations)
  float* gscr = nullptr;               // Gram partials of the second CholeskyQR2 round
  float* Rtmp = nullptr;               // exact path: factor of each product and its inverse (2 rr each)
  float* Rslot = nullptr;              // [2][nprod] lagged factors
  float* Tslot = nullptr;              // [2][nprod] their inverses
  float* Rfin = nullptr;               // Ra, Rb of Q2 and of Q1, each followed by its inverse (2 rr each)
  float* Pi = nullptr;                 // factors applied in the last chain (normalised)
  float* Vprev = nullptr;              // warm start of the core SVD
  Ctl* ctl = nullptr;
  unsigned* cand_key = nullptr;
  long long* cand_idx = nullptr;
  float* cand_val = nullptr;
  unsigned long long cap = 0;
  unsigned* sbits = nullptr;           // two bitmaps of m n bits: the support of the committed S (bitmap
  long long sbits_words = 0;           // ctl->cur) and a clear one the next S-step marks its support in
  size_t sbits_bytes = 0;
  float* XA1 = nullptr;                // m x RP: X A1, the cached part of the first projection (null: the
                                       // first product streams Z)
  long long* S_idx[2] = {nullptr, nullptr};
  float* S_val[2] = {nullptr, nullptr};
  int idx_bits = 1;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // 0 exact path, 1 fast path
  int graph_r[2] = {-1, -1};
  unsigned graph_epoch = 0;   // bumped whenever captured graphs become invalid (buffers, geometry)
  int graph_nodes = 0;
  bool need_exact = true;
  int exact_left = 0;   // exact iterations still owed after an alarm of the lagged normalisers
  int backoff = 1;      // exact iterations owed at the next alarm (doubles while alarms repeat)
  int rank_drops = 0;
  int exact_iters = 0;
  int alarms = 0;          // fast iterations abandoned by a conditioning alarm
  int rescales = 0;
  // kernel-level profiling (eager launches bracketed by events)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> prof_cls;
  std::vector<int> prof_side;   // launch on the side stream
  size_t prof_used = 0;
  // GreBsmo (godec_grebsmo_*): parameters, the borrowed test matrices of the increments
  bool greb = false;
  godec_grebsmo_params gp{};
  const float* omega = nullptr;
  // naive GoDec (godec_naive_init): the L-step is a truncated SVD by subspace iteration
  // over np_cols columns (rank + oversampling), warm-started from the last iteration's basis
  bool naive = false;
  int np_cols = 0;
  // LinGoDec (godec_lingodec_*): the item features' basis Qf = orth(F) (in Q2, d columns),
  // its factors in Rf (R1, R1^{-1}, R2, R2^{-1}), the soft threshold lambda
  bool lingo = false;
  int lg_d = 0;
  double lg_lambda = 0.0;
  char err[200] = {0};
};

static void prof_mark(godec_ctx* c, int cls, cudaStream_t s) {
  if (c->prof_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[c->prof_used++], s);
  if (cls >= 0) {
    c->prof_cls.push_back(cls);
    c->prof_side.push_back(s == c->side_st ? 1 : (s == c->rank_st ? 2 : 0));
  }
}

// Bracket one launch with events when profiling (eager mode only).
#define PROF(c, cls, s, stmt)                       \
  do {                                              \
    if ((c)->prof) prof_mark(c, cls, s);            \
    stmt;                                           \
    if ((c)->prof) prof_mark(c, -1, s);             \
  } while (0)

namespace {

const char* kStatusNames[] = {"ok", "invalid argument", "CUDA error", "out of memory",
                              "non-finite values", "device wait timed out", "invalid state",
                              "unsupported"};

char g_static_err[256];

godec_status fail(godec_ctx* c, godec_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(c, e_ == cudaErrorMemoryAllocation ? GODEC_ERR_OOM : GODEC_ERR_CUDA,    \
                  "%s: %s", #call, cudaGetErrorString(e_));                              \
  } while (0)

int round_up(int v, int a) { return (v + a - 1) / a * a; }

template <typename T>
cudaError_t dalloc(T** p, size_t elems) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(elems, 1) * sizeof(T));
}

void free_graphs(godec_ctx* c) {
  ++c->graph_epoch;
  for (int k = 0; k < 2; ++k) {
    if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
    c->gexec[k] = nullptr;
    c->graph_r[k] = -1;
  }
}

godec_status alloc_candidates(godec_ctx* c, unsigned long long cap) {
  cudaFree(c->cand_key);
  cudaFree(c->cand_idx);
  cudaFree(c->cand_val);
  c->cand_key = nullptr;
  c->cand_idx = nullptr;
  c->cand_val = nullptr;
  c->cap = cap;
  CK(dalloc(&c->cand_key, cap));
  CK(dalloc(&c->cand_idx, cap));
  CK(dalloc(&c->cand_val, cap));
  return GODEC_OK;
}

// ---------------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------------
void fork_side(godec_ctx* c) {
  cudaEvent_t e = c->ev[c->ev_used++ % kEvents];
  cudaEventRecord(e, c->st);
  cudaStreamWaitEvent(c->side_st, e, 0);
}

void join_side(godec_ctx* c) {
  cudaEvent_t e = c->ev[c->ev_used++ % kEvents];
  cudaEventRecord(e, c->side_st);
  cudaStreamWaitEvent(c->st, e, 0);
}

// The rank test runs on a stream of its own: its verdict (a rank drop abandons the
// iteration) is needed only before the S-step commits, so it overlaps the rest of the
// chain instead of delaying the lagged-normaliser updates queued behind it.
void fork_rank(godec_ctx* c) {
  cudaEvent_t e = c->ev[c->ev_used++ % kEvents];
  cudaEventRecord(e, c->st);
  cudaStreamWaitEvent(c->rank_st, e, 0);
  c->rank_forked = true;
}

void join_rank(godec_ctx* c) {
  if (!c->rank_forked) return;
  cudaEvent_t e = c->ev[c->ev_used++ % kEvents];
  cudaEventRecord(e, c->rank_st);
  cudaStreamWaitEvent(c->st, e, 0);
  c->rank_forked = false;
}

char* gpart(godec_ctx* c, int i) { return c->gparts + (size_t)i * c->gpart_stride; }
void* bt2(godec_ctx* c, int b) { return static_cast<char*>(c->bt2) + (size_t)b * 2 * c->RP * c->ldb * 2; }

// The float16 copies of the working matrices (precision form), from Z and Z^T.
void refresh_z16(godec_ctx* c) {
  if (!c->Z16) return;
  launch_to_half(c->Z, c->p.m, c->p.n, c->ldz, c->Z16, c->ldz, c->nsm, c->st);
  launch_to_half(c->Zt, c->p.n, c->p.m, c->ldzt, c->Zt16, c->ldzt, c->nsm, c->st);
}
double* g64(godec_ctx* c, int i) { return c->g64 + (size_t)i * c->RP * c->RP; }
// The float copy of a Gram in c->g64 (written by the same Gram sum), else null.
float* g32_of(godec_ctx* c, const double* g) {
  const size_t n = (size_t)(c->nprod + 2) * c->RP * c->RP;
  return (c->g32 && g >= c->g64 && g < c->g64 + n) ? c->g32 + (g - c->g64) : nullptr;
}

// Product i of the chain: even i streams Z (rows m, K n), odd i streams Z^T (rows n, K m).
// Its skinny operand is the split transposed output of product i-1 (A1 for i = 0); the
// rows go to `out` (nullable) and, with want_bt2, to the operand of product i+1.
void prod(godec_ctx* c, int i, float* out, bool want_bt2, const float* T0, const float* T1, int gram_mode) {
  const bool even = (i % 2) == 0;
  TcLaunch l{};
  l.mapA = c->tmap[even ? 0 : 1];
  l.mapB = c->tmap[i == 0 ? 4 : 2 + ((i - 1) & 1)];
  if (c->Z16) {   // precision form: the chain streams the float16 copies
    l.half_a = 1;
    l.mapA = c->tmap[even ? 8 : 9];   // same two-term operand maps as the float32 chain
  }
  l.rows = even ? c->p.m : c->p.n;
  l.K = even ? c->p.n : c->p.m;
  l.RP = c->RP;
  l.geom = c->tg[even ? 0 : 1];
  l.part = c->part;
  l.counters = c->counters;
  l.out = out;
  l.bt2 = want_bt2 ? bt2(c, i & 1) : nullptr;
  l.ldb = c->ldb;
  l.Tn[0] = T0;
  l.Tn[1] = T1;
  l.cscale = c->cs + (i == 0 ? 0 : c->RP);
  l.zscale = c->ctl->zscale;
  l.prescaled = 1;   // Z and Z^T are stored as (X - S) s_Z
  l.gram_part = gpart(c, i);
  l.gram_mode = gram_mode;
  l.t_upper = 1;     // slot normalisers are inverses of upper-triangular factors
  l.pend = c->pend;
  l.ctl = c->ctl;
  l.pdl = 1;
  l.z_prefetch = i > 0;   // within the chain no kernel writes Z (the S-step comes before product 0)
  PROF(c, 0, c->st, launch_prod_tc(l, c->st));
}

cudaEvent_t record(godec_ctx* c, cudaStream_t s) {
  cudaEvent_t e = c->ev[c->ev_used++ % kEvents];
  cudaEventRecord(e, s);
  return e;
}

void gram_sum(godec_ctx* c, const void* part, int dbl, int64_t nblk, double* out, cudaStream_t s) {
  PROF(c, 1, s, launch_gram_sum(part, dbl, nblk, c->RP, out, c->ctl, s, g32_of(c, out)));
}

// R with Rᵀ R = Gram, and T = R^{-1} stored right after R.
void chol(godec_ctx* c, const double* g, float* R, float alarm_ratio = 0.f) {
  PROF(c, 2, c->st, launch_chol(g, c->r, c->RP, R, R + (size_t)c->RP * c->RP, c->ctl, c->st, alarm_ratio,
                                (c->p.flags & GODEC_FLAG_FP64_FACTOR) != 0, g32_of(c, g)));
}
const float* inv_of(godec_ctx* c, const float* R) { return R + (size_t)c->RP * c->RP; }

void apply(godec_ctx* c, const float* P, int64_t rows, const float* T0, const float* T1, float* Q, float* gram,
           void* bt2out = nullptr) {
  PROF(c, 3, c->st, launch_apply(P, rows, c->RP, T0, T1, Q, gram, c->ctl, c->st, bt2out, c->ldb));
}

// Exact CholeskyQR2 of c->P (rows x RP) with the first-pass Gram g1: Q = P Ra^{-1} Rb^{-1},
// written to fin and, if bt2out is set, as the next product's operand.  With both null the
// last apply is left out: c->P then holds P Ra^{-1} and Q = c->P Rb^{-1} is never formed
// (the last chain product: its Rb^{-1} is folded into the core SVD's left factor).
void final_cqr2(godec_ctx* c, int64_t rows, const double* g1, float* Ra, float* Rb, float* fin, double* g2,
                void* bt2out) {
  chol(c, g1, Ra);
  apply(c, c->P, rows, inv_of(c, Ra), inv_of(c, Ra), c->P, c->gscr);
  gram_sum(c, c->gscr, 0, apply_blocks(rows), g2, c->st);
  chol(c, g2, Rb);
  if (fin || bt2out) apply(c, c->P, rows, inv_of(c, Rb), inv_of(c, Rb), fin, nullptr, bt2out);
}

void slot(godec_ctx* c, SlotLaunch& sl) {
  sl.g32 = g32_of(c, sl.g64);
  sl.r = c->r;
  sl.RP = c->RP;
  sl.ctl = c->ctl;
  sl.alarm_ratio = kAlarmRatio;
  PROF(c, 4, c->side_st, launch_slot(sl, c->side_st));
}

// ---------------------------------------------------------------------------------
// Precision form: one float32 correction of the L factors from the float16 chain
// (reading of the error control for the rounded chain).  With U, V orthonormal, one
// float32-accurate visit of Z and of Z^T gives A = Z V and B = Z^T U; the tangent-space
// correction P_U Z + Z P_V - P_U Z P_V = [U A] K [V B]^T, K = [[-C, I], [I, 0]],
// C = U^T A, is re-truncated to rank r: CholeskyQR2 of [U A] and [V B], SVD of the
// 2r x 2r core.  An error theta of the chain's subspaces moves the corrected L by about
// theta sigma_{r+1} (the residual's spectral norm) instead of theta sigma_1: second order
// when Z - L* is small, a reduction by sigma_{r+1} / sigma_1 otherwise.
// ---------------------------------------------------------------------------------
void cqr2(godec_ctx* c, const float* W, int64_t rows, int R2, int ld, float* Q, float* R1, float* T1, float* R2m,
          float* T2) {
  cudaStream_t st = c->st;
  const int* ab = &c->ctl->abort;
  PROF(c, 10, st, launch_cross_gram(W, ld, R2, W, ld, R2, rows, c->rf_part, kRefineParts, c->rf_g, ld, st, ab));
  const bool f64 = (c->p.flags & GODEC_FLAG_FP64_FACTOR) != 0;
  PROF(c, 10, st, launch_chol(c->rf_g, R2, ld, R1, T1, c->ctl, st, 0.f, f64));
  PROF(c, 10, st, launch_tall_small_f(W, ld, R2, T1, ld, 0, R2, rows, 1.f, 0.f, c->Qtmp, ld, st, ab));
  PROF(c, 10, st, launch_cross_gram(c->Qtmp, ld, R2, c->Qtmp, ld, R2, rows, c->rf_part, kRefineParts, c->rf_g, ld, st, ab));
  PROF(c, 10, st, launch_chol(c->rf_g, R2, ld, R2m, T2, c->ctl, st, 0.f, f64));
  PROF(c, 10, st, launch_tall_small_f(c->Qtmp, ld, R2, T2, ld, 0, R2, rows, 1.f, 0.f, Q, ld, st, ab));
}

void refine(godec_ctx* c) {
  const int r = c->r, RP = c->RP, R2 = 2 * r, ld = (R2 + 7) / 8 * 8;
  const int64_t m = c->p.m, n = c->p.n;
  cudaStream_t st = c->st;
  const int* ab = &c->ctl->abort;   // an abandoned iteration skips the correction too
  // A = Z V, B = Z^T U (float32 product kernel on the float32 working copies)
  TcLaunch l{};
  l.RP = RP;
  l.part = c->part;
  l.counters = c->counters;
  l.cscale = c->cs_ref;
  l.zscale = c->ctl->zscale;
  l.prescaled = 1;
  l.pend = c->pend;
  l.ctl = c->ctl;
  launch_split_t(c->V, n, RP, bt2(c, 3), c->ldb, c->cs_ref, st, ab);
  l.mapA = c->tmap[0];
  l.mapB = c->tmap[13];
  l.rows = m;
  l.K = n;
  l.geom = c->tg[0];
  l.out = c->RA;
  PROF(c, 0, st, launch_prod_tc(l, st));
  launch_split_t(c->U, m, RP, bt2(c, 3), c->ldb, c->cs_ref, st, ab);
  l.mapA = c->tmap[1];
  l.mapB = c->tmap[14];
  l.rows = n;
  l.K = m;
  l.geom = c->tg[1];
  l.out = c->RB;
  PROF(c, 0, st, launch_prod_tc(l, st));
  // C = U^T A; [U A], [V B] (stride ld, zero padding)
  PROF(c, 10, st, launch_cross_gram(c->U, RP, r, c->RA, RP, r, m, c->rf_part, kRefineParts, c->rf_C, r, st, ab));
  PROF(c, 10, st, launch_concat2(c->U, c->RA, RP, r, m, c->Wa, ld, st, ab));
  PROF(c, 10, st, launch_concat2(c->V, c->RB, RP, r, n, c->Wb, ld, st, ab));
  const size_t q = (size_t)64 * 64;
  float *Ra1 = c->Rf, *Ta1 = Ra1 + q, *Ra2 = Ta1 + q, *Ta2 = Ra2 + q, *Rb1 = Ta2 + q, *Tb1 = Rb1 + q,
        *Rb2 = Tb1 + q, *Tb2 = Rb2 + q;
  cqr2(c, c->Wa, m, R2, ld, c->Qa, Ra1, Ta1, Ra2, Ta2);
  cqr2(c, c->Wb, n, R2, ld, c->Qb, Rb1, Tb1, Rb2, Tb2);
  PROF(c, 10, st, launch_refine_core(Ra1, Ra2, Rb1, Rb2, ld, c->rf_C, r, c->rf_core, st, ab));
  PROF(c, 10, st, launch_svd_small(c->rf_core, R2, r, c->rf_U, c->sigma, c->rf_V, st, ab));
  PROF(c, 10, st, launch_tall_small_d(c->Qa, ld, R2, c->rf_U, r, 0, r, m, 1.f, 0.f, c->U, RP, st, ab));
  PROF(c, 10, st, launch_tall_small_d(c->Qb, ld, R2, c->rf_V, r, 0, r, n, 1.f, 0.f, c->V, RP, st, ab));
}

// ---------------------------------------------------------------------------------
// L-step of Algorithm 1 (power chain, rank test, core and root)
// ---------------------------------------------------------------------------------
void enqueue_lstep(godec_ctx* c, bool fast) {
  const int q = c->p.q, RP = c->RP;
  const int64_t m = c->p.m, n = c->p.n;
  const int nprod = c->nprod, i_q2 = 4 * q + 1, i_rank = 4 * q + 2, last = nprod - 1;
  const size_t rr = (size_t)RP * RP;
  auto sR = [&](int h, int i) { return c->Rslot + ((size_t)h * nprod + i) * rr; };
  auto sT = [&](int h, int i) { return c->Tslot + ((size_t)h * nprod + i) * rr; };
  const float* rapp_last[2] = {nullptr, nullptr};
  bool have_pi = false;
  cudaEvent_t rank_gram = nullptr;                // the rank test's Gram of P (fast path)
  cudaEvent_t side_core = nullptr;                // side work the core SVD needs (all but the last slot)
  for (int i = 0; i < nprod; ++i) {
    const bool even = (i % 2) == 0;
    const int64_t rows = even ? m : n;
    const int64_t tiles = prod_tiles(rows);
    void* nextB = bt2(c, i & 1);
    // the rank test's Gram reads P until `last` rewrites it
    if (i == last && rank_gram) {
      cudaStreamWaitEvent(c->st, rank_gram, 0);
      rank_gram = nullptr;
    }
    SlotLaunch sl;
    sl.R_next[0] = sR(0, i);
    sl.R_next[1] = sR(1, i);
    sl.T_next[0] = sT(0, i);
    sl.T_next[1] = sT(1, i);
    sl.Pi = c->Pi;
    const int pi_mode = (i == i_rank) ? 2 : ((i > i_rank && i < last) ? 1 : 0);
    sl.pi_mode = pi_mode;
    if (i == i_rank) {
      // P = Z Q2 unnormalised, with an exactly accumulated Gram for the rank test.  On the
      // fast path nothing on the critical path needs that Gram: it is formed on the rank
      // test's stream from P instead of in the product's tile completion.
      const bool aside = fast && i != last;
      prod(c, i, c->P, false, nullptr, nullptr, aside ? 0 : 2);
      if (aside) {
        fork_rank(c);
        PROF(c, 1, c->rank_st, launch_gram_tiles(c->P, rows, RP, 2, gpart(c, i), c->ctl, c->rank_st));
        gram_sum(c, gpart(c, i), 1, tiles, g64(c, i), c->rank_st);
        rank_gram = record(c, c->rank_st);
      } else {
        gram_sum(c, gpart(c, i), 1, tiles, g64(c, i), c->st);
        fork_rank(c);
      }
      PROF(c, 5, c->rank_st,
           launch_rank(g64(c, i), c->r, RP, c->p.rank_tol > 0 ? c->p.rank_tol : 1e-4, c->ctl, c->rank_st));
      if (i == last) {   // q = 0: this product is also the last one
        final_cqr2(c, rows, g64(c, i), c->Rfin + 4 * rr, c->Rfin + 6 * rr, nullptr, g64(c, nprod + 1), nullptr);
        continue;
      }
      if (fast) {
        apply(c, c->P, rows, sT(0, i), sT(1, i), nullptr, nullptr, nextB);
        cudaStreamWaitEvent(c->side_st, rank_gram, 0);   // the slot update reads that Gram
        sl.fast = 1;
        sl.g64 = g64(c, i);
        sl.g_is_p = 1;
        sl.R_app[0] = sR(0, i);
        sl.R_app[1] = sR(1, i);
        sl.T_app[0] = sT(0, i);
        sl.T_app[1] = sT(1, i);
      } else {
        float* Rt = c->Rtmp + (size_t)i * 2 * rr;
        chol(c, g64(c, i), Rt);
        apply(c, c->P, rows, inv_of(c, Rt), inv_of(c, Rt), nullptr, nullptr, nextB);
        fork_side(c);
        sl.fast = 0;
        sl.R_app[0] = sl.R_app[1] = Rt;
      }
      slot(c, sl);
      have_pi = true;
    } else if (i == i_q2 || i == last) {
      prod(c, i, c->P, false, fast ? sT(0, i) : nullptr, fast ? sT(1, i) : nullptr, 1);
      gram_sum(c, gpart(c, i), 0, tiles, g64(c, i), c->st);
      float* Ra = c->Rfin + (i == i_q2 ? 0 : 4) * rr;
      float* Rb = Ra + 2 * rr;
      // Q1 (the last product's basis) is never formed: U = Q1 Um = P (R^{-1} Um) with the
      // factor's inverse folded into the core SVD's output
      float* fin = (i == i_q2) ? c->Q2 : nullptr;
      if (fast) {
        // the lagged normaliser left P almost orthonormal: one CholeskyQR pass
        chol(c, g64(c, i), Ra, kCqr1Ratio);
        if (i == i_q2) apply(c, c->P, rows, inv_of(c, Ra), inv_of(c, Ra), fin, nullptr, nextB);
        Rb = nullptr;
      } else {
        final_cqr2(c, rows, g64(c, i), Ra, Rb, fin, g64(c, nprod + (i == i_q2 ? 0 : 1)),
                   i == i_q2 ? nextB : nullptr);
      }
      // the last slot update prepares the next iteration only: the core SVD waits for the
      // side work queued before it, not for it
      if (i == last) side_core = record(c, c->side_st);
      fork_side(c);
      sl.fast = 0;
      if (fast) {
        sl.R_app[0] = sR(0, i);
        sl.R_app[1] = sR(1, i);
        if (i == last) {
          rapp_last[0] = sR(0, i);
          rapp_last[1] = sR(1, i);
        }
      }
      sl.L1 = Ra;
      sl.L2 = Rb;   // null after a single pass
      sl.pi_mode = 0;
      slot(c, sl);
    } else {
      // the first projection (X - S) A1 = X A1 - S A1 from the cached X A1
      const bool sp = i == 0 && c->XA1;
      if (sp)
        PROF(c, 11, c->st,
             launch_sproj(c->XA1, c->A1, RP, c->X, c->p.ldx, c->Z, c->ldz, m, n, c->sbits, c->sbits_words, c->ctl,
                          c->P, c->st));
      if (fast && sp) {
        apply(c, c->P, rows, sT(0, i), sT(1, i), nullptr, c->gscr, nextB);
        fork_side(c);
        gram_sum(c, c->gscr, 0, apply_blocks(rows), g64(c, i), c->side_st);
        sl.fast = 1;
        sl.g64 = g64(c, i);
        sl.R_app[0] = sR(0, i);
        sl.R_app[1] = sR(1, i);
      } else if (fast) {
        // (the lagged normaliser's Gram stays in the tile completion: the side stream runs
        // on the few SMs the product leaves free and has no room for it)
        prod(c, i, nullptr, true, sT(0, i), sT(1, i), 1);
        fork_side(c);
        gram_sum(c, gpart(c, i), 0, tiles, g64(c, i), c->side_st);
        sl.fast = 1;
        sl.g64 = g64(c, i);
        sl.R_app[0] = sR(0, i);
        sl.R_app[1] = sR(1, i);
      } else {
        float* Rt = c->Rtmp + (size_t)i * 2 * rr;
        if (sp) PROF(c, 1, c->st, launch_gram_tiles(c->P, rows, RP, 1, gpart(c, i), c->ctl, c->st));
        else prod(c, i, c->P, false, nullptr, nullptr, 1);
        gram_sum(c, gpart(c, i), 0, tiles, g64(c, i), c->st);
        chol(c, g64(c, i), Rt);
        apply(c, c->P, rows, inv_of(c, Rt), inv_of(c, Rt), nullptr, nullptr, nextB);
        fork_side(c);
        sl.fast = 0;
        sl.R_app[0] = sl.R_app[1] = Rt;
      }
      slot(c, sl);
      if (pi_mode) have_pi = true;
    }
  }
  if (side_core) cudaStreamWaitEvent(c->st, side_core, 0);
  else join_side(c);
  // r x r core, SVD and singular-value root, then L = (Q1 Um) diag(sigma) (Q2 Vm)^T with
  // Q1 Um = P (Rl^{-1} Um), Rl the last factor applied to P (Ra after one CholeskyQR pass,
  // Rb after two): the SVD kernel returns Rl^{-1} Um; V is formed on the rank test's
  // stream (long idle by then; the side stream may still run the last slot update)
  const float* Rb_last = (fast && last != i_rank) ? nullptr : c->Rfin + 6 * rr;
  const float* Tl = inv_of(c, Rb_last ? Rb_last : c->Rfin + 4 * rr);
  PROF(c, 6, c->st,
       launch_svd(c->Rfin + 4 * rr, Rb_last, rapp_last[0], rapp_last[1], have_pi ? c->Pi : nullptr,
                  c->Vprev, c->r, RP, q, c->Um, c->Vm, c->sigma, c->ctl, c->st, Tl));
  fork_rank(c);
  PROF(c, 3, c->rank_st, launch_apply(c->Q2, n, RP, c->Vm, c->Vm, c->V, nullptr, c->ctl, c->rank_st));
  apply(c, c->P, m, c->Um, c->Um, c->U, nullptr);
  join_rank(c);
  if (c->Z16 && !(c->p.flags & GODEC_FLAG_NO_REFINE)) refine(c);
  // operands of the tensor-core residual pass
  PROF(c, 3, c->st, launch_lsplit(c->U, c->V, c->sigma, m, n, RP, c->r, c->ctl->zscale, c->LA, c->LB, c->st));
  join_side(c);
}

// S-step of one iteration (Algorithm 1, eq. raw_lss) on the current L factors; r = 0 means L = 0.
void enqueue_sstep(godec_ctx* c, int r) {
  const int64_t m = c->p.m, n = c->p.n;
  cudaStream_t st = c->st;
  ResidualArgs ra{};
  ra.X = c->X;
  ra.m = m;
  ra.n = n;
  ra.ldx = c->p.ldx;
  ra.U = c->U;
  ra.sigma = c->sigma;
  ra.V = c->V;
  ra.r = r;
  ra.RP = c->RP;
  ra.ctl = c->ctl;
  ra.cand_key = c->cand_key;
  ra.cand_idx = c->cand_idx;
  ra.cand_val = c->cand_val;
  ra.cand_cap = c->cap;
  for (int pass = 0; pass < 3; ++pass) {
    ra.pass = pass;
    if (c->LA && r > 0) {
      ResidTcLaunch rl{};
      rl.ra = ra;
      rl.mapX = c->tmap[5];
      rl.mapA = c->tmap[6];
      rl.mapB = c->tmap[7];
      rl.zscale = c->ctl->zscale;
      rl.nsm = c->nsm;
      PROF(c, 7, st, launch_resid_tc(rl, st));
    } else {
      PROF(c, 7, st, launch_residual(ra, c->nsm, st));
    }
    PROF(c, 8, st, launch_after_pass(c->ctl, pass, c->p.k, c->cap, st));
  }
  SelectArgs se{};
  se.ctl = c->ctl;
  se.cand_key = c->cand_key;
  se.cand_idx = c->cand_idx;
  se.cand_val = c->cand_val;
  se.cand_cap = c->cap;
  se.k = c->p.k;
  se.idx_bits = c->idx_bits;
  for (int round = 0; round < 7; ++round) {
    se.round = round;
    PROF(c, 8, st, launch_select_round(se, c->nsm, st));
  }
  EmitArgs ea{};
  ea.ctl = c->ctl;
  ea.cand_key = c->cand_key;
  ea.cand_idx = c->cand_idx;
  ea.cand_val = c->cand_val;
  ea.cand_cap = c->cap;
  ea.S_idx[0] = c->S_idx[0];
  ea.S_idx[1] = c->S_idx[1];
  ea.S_val[0] = c->S_val[0];
  ea.S_val[1] = c->S_val[1];
  ea.X = c->X;
  ea.n = n;
  ea.ldx = c->p.ldx;
  ea.Z = c->Z;
  ea.ldz = c->ldz;
  ea.Zt = c->Zt;
  ea.ldzt = c->ldzt;
  ea.Z16 = c->Z16;
  ea.Zt16 = c->Zt16;
  ea.zscale = c->ctl->zscale;
  ea.max_nnz = c->p.k;
  ea.sbits = c->sbits;
  ea.sbits_words = c->sbits_words;
  PROF(c, 8, st, launch_emit(ea, c->nsm, st));
  if (c->Z) PROF(c, 9, st, launch_z_update(ea, c->nsm, st));
}

// Product over Z (even: m rows, K = n) or Z^T (odd: n rows, K = m) with the operand of
// tensor map map_b, its column scales cscale, Gram partials into slot gslot (gram_mode 1).
void greb_prod(godec_ctx* c, bool even, int map_b, const float* cscale, float* out, int gram_mode, int gslot) {
  TcLaunch l{};
  l.mapA = c->tmap[even ? 0 : 1];
  l.mapB = c->tmap[map_b];
  l.rows = even ? c->p.m : c->p.n;
  l.K = even ? c->p.n : c->p.m;
  l.RP = c->RP;
  l.geom = c->tg[even ? 0 : 1];
  l.part = c->part;
  l.counters = c->counters;
  l.out = out;
  l.ldb = c->ldb;
  l.cscale = cscale;
  l.zscale = c->ctl->zscale;
  l.prescaled = 1;
  l.gram_part = gpart(c, gslot);
  l.gram_mode = gram_mode;
  l.t_upper = 1;
  l.pend = c->pend;
  l.ctl = c->ctl;
  launch_prod_tc(l, c->st);
}

// out (m x RP) = D B with D = Z - U W^T (the derivative of eq. GreBsmoD; U = 0 at rank 0);
// B (n x RP) has p nonzero columns.
void greb_apply_D(godec_ctx* c, int ri, int p, const float* B, float* out) {
  const int RP = c->RP;
  launch_split_t(B, c->p.n, RP, bt2(c, 3), c->ldb, c->cs_ref, c->st, &c->ctl->abort);
  greb_prod(c, true, 13, c->cs_ref, out, 0, 0);
  if (ri > 0) {
    launch_cross_gram(c->Q2, RP, ri, B, RP, p, c->p.n, c->rf_part, kRefineParts, c->rf_C, RP, c->st, &c->ctl->abort);
    launch_tall_small_d(c->Q1, RP, ri, c->rf_C, RP, 0, p, c->p.m, -1.f, 1.f, out, RP, c->st, &c->ctl->abort);
  }
}

// out (n x RP) = D^T Y for Y (m x RP) with p nonzero columns.
void greb_apply_Dt(godec_ctx* c, int ri, int p, const float* Y, float* out) {
  const int RP = c->RP;
  launch_split_t(Y, c->p.m, RP, bt2(c, 3), c->ldb, c->cs_ref, c->st, &c->ctl->abort);
  greb_prod(c, false, 14, c->cs_ref, out, 0, 0);
  if (ri > 0) {
    launch_cross_gram(c->Q1, RP, ri, Y, RP, p, c->p.m, c->rf_part, kRefineParts, c->rf_C, RP, c->st, &c->ctl->abort);
    launch_tall_small_d(c->Q2, RP, ri, c->rf_C, RP, 0, p, c->p.n, -1.f, 1.f, out, RP, c->st, &c->ctl->abort);
  }
}

// L-step of naive GoDec (eq. raw_lss: L = the rank-r truncated SVD of Z = X - S) by block
// subspace iteration over np_cols = r + oversampling columns: from the basis B the last
// iteration ended with, q times B = orth(Z^T orth(Z B)), then the Rayleigh-Ritz step
// Z B = Qa R, R = Ur S Vr^T, L = (Qa Ur) S (B Vr)^T truncated to r (float64 SVD of R).
void enqueue_naive_lstep(godec_ctx* c) {
  const int RP = c->RP, p = c->np_cols, r = c->r;
  const int64_t m = c->p.m, n = c->p.n;
  cudaStream_t st = c->st;
  const size_t q = (size_t)64 * 64;
  float *R1 = c->Rf, *T1 = R1 + q, *R2m = T1 + q, *T2 = R2m + q;
  for (int s = 0; s < c->p.q; ++s) {
    greb_apply_D(c, 0, p, c->Qb, c->P);
    cqr2(c, c->P, m, p, RP, c->Qa, R1, T1, R2m, T2);
    greb_apply_Dt(c, 0, p, c->Qa, c->P);
    cqr2(c, c->P, n, p, RP, c->Qb, R1, T1, R2m, T2);
  }
  greb_apply_D(c, 0, p, c->Qb, c->P);
  cqr2(c, c->P, m, p, RP, c->Qa, R1, T1, R2m, T2);
  const int* ab = &c->ctl->abort;   // an abandoned iteration leaves U, V and the basis as they were
  launch_rmul(R2m, R1, RP, p, c->rf_core, 0, nullptr, st, ab);
  launch_svd_small(c->rf_core, p, r, c->rf_U, c->sigma, c->rf_V, st, ab, true);
  launch_tall_small_d(c->Qa, RP, p, c->rf_U, r, 0, r, m, 1.f, 0.f, c->U, RP, st, ab);
  launch_tall_small_d(c->Qb, RP, p, c->rf_V, r, 0, r, n, 1.f, 0.f, c->V, RP, st, ab);
  launch_lsplit(c->U, c->V, c->sigma, m, n, RP, r, c->ctl->zscale, c->LA, c->LB, st, ab);
}

void enqueue_iteration(godec_ctx* c, bool fast) {
  if (c->naive) {
    enqueue_naive_lstep(c);
    enqueue_sstep(c, c->r);
    return;
  }
  enqueue_lstep(c, fast);
  enqueue_sstep(c, c->r);
}

godec_status build_graph(godec_ctx* c, int mode) {
  if (c->gexec[mode]) cudaGraphExecDestroy(c->gexec[mode]);
  c->gexec[mode] = nullptr;
  cudaGraph_t g = nullptr;
  // The caller's stream may be the legacy default stream, which cannot be captured:
  // record on a private stream and launch the graph on the caller's stream.
  CK(cudaStreamSynchronize(c->st));
  cudaStream_t user = c->st;
  c->st = c->cap_st;
  cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_iteration(c, mode == 1);
    e = cudaStreamEndCapture(c->st, &g);
  }
  c->st = user;
  if (e != cudaSuccess) return fail(c, GODEC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  e = cudaGraphInstantiate(&c->gexec[mode], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, GODEC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graph_r[mode] = c->r;
  if (mode == 1) c->graph_nodes = (int)nodes;
  return GODEC_OK;
}

godec_status read_ctl(godec_ctx* c, Ctl* h) {
  CK(cudaMemcpyAsync(h, c->ctl, offsetof(Ctl, hist), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

template <typename T>
godec_status set_field(godec_ctx* c, size_t off, T v) {
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(c->ctl) + off, &v, sizeof(T), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}
#define SET_CTL(field, v) set_field(c, offsetof(Ctl, field), (decltype(Ctl::field))(v))

// After the rank test lowered r: keep only the first r columns of A1 (reading of
// "r := rank(A2^T Y1)"), so every product of the chain has zero columns beyond r.
godec_status drop_columns(godec_ctx* c) {
  if (c->r < c->RP)
    CK(cudaMemset2DAsync(c->A1 + c->r, c->RP * sizeof(float), 0, (c->RP - c->r) * sizeof(float), c->p.n,
                         c->st));
  launch_split_t(c->A1, c->p.n, c->RP, bt2(c, 2), c->ldb, c->cs, c->st);
  // X A1 loses the same columns (the others keep their split scales, so this is exactly
  // the product over the new A1)
  if (c->XA1 && c->r < c->RP)
    CK(cudaMemset2DAsync(c->XA1 + c->r, c->RP * sizeof(float), 0, (c->RP - c->r) * sizeof(float), c->p.m,
                         c->st));
  return GODEC_OK;
}

// Both support bitmaps cleared, then the committed S's support marked again in bitmap
// ctl->cur (an S-step cut short may have marked entries in the other one).
godec_status rebuild_sbits(godec_ctx* c) {
  if (!c->sbits) return GODEC_OK;
  CK(cudaMemsetAsync(c->sbits, 0, c->sbits_bytes, c->st));
  launch_sbits_rebuild(c->sbits, c->sbits_words, c->S_idx, c->ctl, c->p.k, c->st);
  CK(cudaGetLastError());
  return GODEC_OK;
}

// X A1 for the chain's first projection (k_sproj.cu): the tensor-core product over X
// itself, split at Z's scale s_Z (set from max |X|, so X s_Z stays in the split's range).
void form_xa1(godec_ctx* c) {
  TcLaunch l{};
  l.mapA = c->tmap[5];
  l.mapB = c->tmap[4];
  l.rows = c->p.m;
  l.K = c->p.n;
  l.RP = c->RP;
  l.geom = c->tg[0];
  l.part = c->part;
  l.counters = c->counters;
  l.out = c->XA1;
  l.cscale = c->cs;
  l.zscale = c->ctl->zscale;
  l.prescaled = 0;
  l.pend = c->pend;
  l.ctl = c->ctl;
  launch_prod_tc(l, c->st);
}

// A product that saw the abort flag part-way leaves tile counters behind.
godec_status clear_counters(godec_ctx* c) {
  CK(cudaMemsetAsync(c->counters, 0, (size_t)c->ncounters * sizeof(unsigned), c->st));
  return GODEC_OK;
}

godec_status reset_state(godec_ctx* c) {
  free_graphs(c);
  c->r = c->p.r;
  c->rank_drops = 0;
  c->need_exact = true;
  c->exact_left = 0;
  c->backoff = 1;
  c->exact_iters = 0;
  c->alarms = 0;
  CK(cudaMemcpyAsync(c->A1, c->A1_orig, (size_t)c->p.n * c->RP * sizeof(float), cudaMemcpyDeviceToDevice,
                     c->st));
  launch_split_t(c->A1, c->p.n, c->RP, bt2(c, 2), c->ldb, c->cs, c->st);
  if (godec_status s = clear_counters(c)) return s;
  std::vector<float> eye((size_t)c->RP * c->RP, 0.f);
  for (int i = 0; i < c->RP; ++i) eye[(size_t)i * c->RP + i] = 1.f;
  CK(cudaMemcpyAsync(c->Vprev, eye.data(), eye.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
  Ctl h;
  memset(&h, 0, offsetof(Ctl, hist));
  h.k_req = c->p.k;
  h.k_eff = c->p.k;
  h.r_eff = c->p.r;
  h.tol = -1.0;
  CK(cudaMemcpyAsync(c->ctl, &h, offsetof(Ctl, hist), cudaMemcpyHostToDevice, c->st));
  if (godec_status s = rebuild_sbits(c)) return s;   // S = 0: both bitmaps empty
  launch_sumsq(c->X, c->p.m, c->p.n, c->p.ldx,
               reinterpret_cast<double*>(reinterpret_cast<char*>(c->ctl) + offsetof(Ctl, normX2)), c->nsm, c->st);
  // working copies Z = X s_Z and Z^T, with s_Z from max |X|
  launch_zscale(c->X, c->p.m, c->p.n, c->p.ldx, &c->ctl->zmax_bits, c->ctl->zscale, c->nsm, c->st);
  launch_scale_copy(c->X, c->p.m, c->p.n, c->p.ldx, c->Z, c->ldz, c->ctl->zscale, c->nsm, c->st);
  launch_transpose(c->X, c->p.m, c->p.n, c->p.ldx, c->Zt, c->ldzt, c->st, c->ctl->zscale);
  refresh_z16(c);
  if (c->XA1) form_xa1(c);
  launch_reset_iter(c->ctl, c->st);
  if (c->lingo) {
    // the features' basis Qf = orth(F) (F was copied into A1) and its split operand, fixed
    // for the whole run; Rf keeps F = Qf R2 R1 for the final W
    const size_t q = (size_t)64 * 64;
    float *R1 = c->Rf, *T1 = R1 + q, *R2m = T1 + q, *T2 = R2m + q;
    launch_fill_zero(c->Q2, (size_t)c->p.n * c->RP * sizeof(float), c->st);
    launch_fill_zero(c->U, (size_t)c->p.m * c->RP * sizeof(float), c->st);
    launch_fill_zero(c->V, (size_t)c->p.n * c->RP * sizeof(float), c->st);
    launch_fill_zero(c->sigma, (size_t)c->RP * sizeof(float), c->st);
    cqr2(c, c->A1, c->p.n, c->lg_d, c->RP, c->Q2, R1, T1, R2m, T2);
    launch_split_t(c->Q2, c->p.n, c->RP, bt2(c, 2), c->ldb, c->cs, c->st);
  }
  if (c->naive) {
    // the first subspace iteration starts from orth(Omega); later ones from the basis the
    // previous iteration ended with
    const size_t q = (size_t)64 * 64;
    float *R1 = c->Rf, *T1 = R1 + q, *R2m = T1 + q, *T2 = R2m + q;
    launch_fill_zero(c->Qb, (size_t)c->p.n * 64 * sizeof(float), c->st);
    launch_fill_zero(c->Qa, (size_t)c->p.m * 64 * sizeof(float), c->st);
    launch_fill_zero(c->U, (size_t)c->p.m * c->RP * sizeof(float), c->st);
    launch_fill_zero(c->V, (size_t)c->p.n * c->RP * sizeof(float), c->st);
    launch_fill_zero(c->sigma, (size_t)c->RP * sizeof(float), c->st);
    cqr2(c, c->A1, c->p.n, c->np_cols, c->RP, c->Qb, R1, T1, R2m, T2);
    // a cold start from a random basis gets kNaiveColdSteps more power steps on X, so the
    // first L-step is as converged as the warm-started ones that follow
    for (int s = 0; s < kNaiveColdSteps; ++s) {
      greb_apply_D(c, 0, c->np_cols, c->Qb, c->P);
      cqr2(c, c->P, c->p.m, c->np_cols, c->RP, c->Qa, R1, T1, R2m, T2);
      greb_apply_Dt(c, 0, c->np_cols, c->Qa, c->P);
      cqr2(c, c->P, c->p.n, c->np_cols, c->RP, c->Qb, R1, T1, R2m, T2);
    }
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

// The S-step wrote an entry of Z beyond the float16 split's range: bring max |Z| back
// into [2^12, 2^13) by a power of two, exactly, in Z, Z^T and the stored scale.
godec_status rescale_z(godec_ctx* c) {
  float* f = c->rescale_tmp;
  launch_zscale(c->Z, c->p.m, c->p.n, c->ldz, &c->ctl->zmax_bits, f, c->nsm, c->st);
  launch_scale_copy(c->Z, c->p.m, c->p.n, c->ldz, c->Z, c->ldz, f, c->nsm, c->st);
  launch_scale_copy(c->Zt, c->p.n, c->p.m, c->ldzt, c->Zt, c->ldzt, f, c->nsm, c->st);
  launch_scale_update(c->ctl->zscale, f, c->st);
  refresh_z16(c);
  CK(cudaGetLastError());
  ++c->rescales;
  return GODEC_OK;
}

// Host-side handling of an aborted iteration; the iteration is redone afterwards.
godec_status handle_abort(godec_ctx* c, const Ctl& h) {
  godec_status s;
  if ((s = clear_counters(c))) return s;
  // an S-step cut short may leave support bits behind
  if ((s = rebuild_sbits(c))) return s;
  if (h.timeout) {
    launch_reset_iter(c->ctl, c->st);
    return fail(c, GODEC_ERR_TIMEOUT, "a bounded device-side wait gave up (iteration %d)", h.iter + 1);
  }
  if (h.range_err && !h.nonfinite) {
    // Z outgrew its scale in the last S-step; the iteration after it was skipped.
    if ((s = rescale_z(c))) return s;
    if ((s = SET_CTL(range_err, 0))) return s;
    launch_reset_iter(c->ctl, c->st);
    CK(cudaGetLastError());
    return GODEC_OK;
  }
  if (h.nonfinite) {
    launch_reset_iter(c->ctl, c->st);
    return fail(c, GODEC_ERR_NONFINITE, "non-finite values in X - L (iteration %d)", h.iter + 1);
  }
  if (h.rank_drop) {
    c->r = h.r_eff;
    ++c->rank_drops;
    c->need_exact = true;
    if (c->r <= 0) return fail(c, GODEC_ERR_UNSUPPORTED, "rank test found rank 0 (X - S is zero)");
    if ((s = drop_columns(c))) return s;
  } else if (h.alarm) {
    ++c->alarms;
    // the lagged normalisers no longer condition the chain (its subspaces moved): stay on
    // the exact path for `backoff` iterations, twice as many at each repeated alarm
    c->need_exact = true;
    c->exact_left = c->backoff;
    c->backoff = std::min(2 * c->backoff, kMaxBackoff);
  } else if (h.need_bigger_cand) {
    unsigned long long cap = c->cap * 2;
    const unsigned long long mn = (unsigned long long)(c->p.m * c->p.n);
    if (cap > mn) cap = mn;
    if (cap <= c->cap) return fail(c, GODEC_ERR_STATE, "candidate buffer cannot grow");
    free_graphs(c);
    if ((s = alloc_candidates(c, cap))) return s;
  } else {
    return fail(c, GODEC_ERR_STATE, "iteration aborted without a reason");
  }
  launch_reset_iter(c->ctl, c->st);
  CK(cudaGetLastError());
  return GODEC_OK;
}

// Path bookkeeping after k completed iterations on the fast (lagged normalisers) or the
// exact path.
void note_done(godec_ctx* c, bool fast, int k) {
  if (k <= 0) return;
  if (fast) {
    c->backoff = 1;
    return;
  }
  c->exact_iters += k;
  c->exact_left -= k;
  if (c->exact_left <= 0) {
    c->exact_left = 0;
    c->need_exact = false;
  }
}

// Run n iterations (graph launches), handling aborted iterations; with tol >= 0 stop early
// on convergence.  The exact path runs whenever the lagged normalisers are not valid.
godec_status run_iterations(godec_ctx* c, int n_iter, double tol) {
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  const int start = h.iter;
  if (h.tol != tol) {
    if ((s = SET_CTL(tol, tol))) return s;
  }
  int guard = 0, done = 0;
  int chunk = tol >= 0.0 ? 1 : n_iter;
  while (done < n_iter) {
    const int mode = c->need_exact ? 0 : 1;
    if (!c->gexec[mode] || c->graph_r[mode] != c->r) {
      if ((s = build_graph(c, mode))) return s;
    }
    const int want = std::min(mode == 0 ? std::max(c->exact_left, 1) : chunk, n_iter - done);
    for (int i = 0; i < want; ++i) CK(cudaGraphLaunch(c->gexec[mode], c->st));
    if ((s = read_ctl(c, &h))) return s;
    const int before = done;
    done = h.iter - start;
    note_done(c, mode == 1, done - before);
    if (h.abort) {
      if (h.converged) return GODEC_OK;
      if ((s = handle_abort(c, h))) return s;
      if (++guard > 64) return fail(c, GODEC_ERR_STATE, "too many aborted iterations");
      continue;
    }
    if (tol >= 0.0 && chunk < 8) chunk *= 2;
  }
  return GODEC_OK;
}

bool bad_params(const godec_params* p, char* why, size_t nwhy) {
  if (!p) { snprintf(why, nwhy, "params is NULL"); return true; }
  if (p->m < 1 || p->n < 1) { snprintf(why, nwhy, "m and n must be >= 1"); return true; }
  if (p->ldx < p->n || (p->ldx * 4) % 16) { snprintf(why, nwhy, "ldx must be >= n and ldx*4 a multiple of 16"); return true; }
  if (p->r < 1 || p->r > GODEC_MAX_RANK || p->r > p->m || p->r > p->n) {
    snprintf(why, nwhy, "r must satisfy 1 <= r <= min(m, n, %d)", GODEC_MAX_RANK); return true;
  }
  if (p->q < 0 || p->q > 8) { snprintf(why, nwhy, "q must be in [0, 8]"); return true; }
  if (p->k < 0 || p->k > p->m * p->n) { snprintf(why, nwhy, "k must be in [0, m*n]"); return true; }
  if (p->max_iter < 1) { snprintf(why, nwhy, "max_iter must be >= 1"); return true; }
  if (p->precision != GODEC_PREC_FP32 && p->precision != GODEC_PREC_BF16_REFINE) {
    snprintf(why, nwhy, "unknown precision"); return true;
  }
  if (p->precision == GODEC_PREC_BF16_REFINE && p->r > 32) {
    snprintf(why, nwhy, "the precision form needs r <= 32"); return true;
  }
  // the S-step's radix histograms count entries in 32 bits
  if ((double)p->m * (double)p->n >= 4294967296.0) { snprintf(why, nwhy, "m*n must be below 2^32"); return true; }
  if ((p->flags & GODEC_FLAG_SPARSE_FIRST) && (p->flags & GODEC_FLAG_DENSE_FIRST)) {
    snprintf(why, nwhy, "GODEC_FLAG_SPARSE_FIRST and GODEC_FLAG_DENSE_FIRST exclude each other"); return true;
  }
  return false;
}

}  // namespace

void godec::set_static_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_static_err, sizeof(g_static_err), fmt, ap);
  va_end(ap);
}

extern "C" {

const char* godec_status_string(godec_status s) {
  int i = (int)s;
  return (i >= 0 && i < 8) ? kStatusNames[i] : "unknown status";
}

const char* godec_last_error(const godec_ctx* c) { return c ? c->err : g_static_err; }

void godec_destroy(godec_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  free_graphs(c);
  void* ptrs[] = {c->Z, c->Zt, c->Z16, c->Zt16, c->A1, c->A1_orig, c->P, c->bt2, c->cs, c->rescale_tmp, c->LA, c->LB, c->Q1, c->Q2,
                  c->U, c->V, c->sigma, c->Um, c->Vm, c->part, c->counters, c->pend, c->gparts, c->RA, c->RB, c->Wa, c->Wb, c->Qa, c->Qb, c->Qtmp, c->Rf,
                  c->cs_ref, c->rf_part, c->rf_g, c->rf_C, c->rf_core, c->rf_U, c->rf_V, c->g64, c->g32, c->gscr,
                  c->Rtmp, c->Rslot, c->Tslot, c->Rfin, c->Pi, c->Vprev, c->ctl, c->cand_key, c->cand_idx,
                  c->cand_val, c->S_idx[0], c->S_idx[1], c->S_val[0], c->S_val[1], c->sbits, c->XA1};
  for (void* p : ptrs) cudaFree(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  if (c->side_st) cudaStreamDestroy(c->side_st);
  if (c->rank_st) cudaStreamDestroy(c->rank_st);
  delete c;
}

// Context set-up shared by GoDec (godec_init) and GreBsmo (godec_grebsmo_init, greb: the
// correction scratch of the precision form and the second skinny-operand maps are also
// allocated, A1 may be NULL).
static godec_status init_ctx(godec_ctx** out, const godec_params* p, const float* X, const float* A1,
                             void* stream, bool greb, int naive_cols = 0, int lingo_d = 0, double lingo_lambda = 0.0) {
  godec_ctx* c = new (std::nothrow) godec_ctx;
  if (!c) return GODEC_ERR_OOM;
  c->greb = greb;
  c->naive = naive_cols > 0;
  c->np_cols = naive_cols;
  c->lingo = lingo_d > 0;
  c->lg_d = lingo_d;
  c->lg_lambda = lingo_lambda;
  c->p = *p;
  c->r = p->r;
  c->RP = round_up(std::max(std::max(p->r, naive_cols), lingo_d), 8);
  c->nprod = 6 * p->q + 3;
  c->st = reinterpret_cast<cudaStream_t>(stream);
  auto bail = [&](godec_status s) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_init: %.200s", c->err);
    godec_destroy(c);
    return s;
  };
#define CKI(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      fail(c, GODEC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));                      \
      return bail(e_ == cudaErrorMemoryAllocation ? GODEC_ERR_OOM : GODEC_ERR_CUDA);         \
    }                                                                                        \
  } while (0)
  CKI(cudaGetDevice(&c->dev));
  CKI(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev));
  c->nsm_dev = c->nsm;
  CKI(prepare_small_kernels());
  CKI(prepare_select_kernels());
  CKI(prepare_stream_kernels());
  CKI(prepare_tc_kernels());
  CKI(prepare_resid_kernels());
  CKI(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  CKI(cudaStreamCreateWithFlags(&c->side_st, cudaStreamNonBlocking));
  CKI(cudaStreamCreateWithFlags(&c->rank_st, cudaStreamNonBlocking));
  for (int k = 0; k < kEvents; ++k) CKI(cudaEventCreateWithFlags(&c->ev[k], cudaEventDisableTiming));
  const int64_t m = p->m, n = p->n, mx = std::max(m, n);
  const int RP = c->RP, np = c->nprod;
  const size_t rr = (size_t)RP * RP;
  c->X = X;
  // rows of the working copies start on 256-byte boundaries: every 128-byte TMA box row
  // is then one whole cache line (a 40000-byte pitch, say, splits every other one)
  c->ldz = (n + 63) / 64 * 64;
  c->ldzt = (m + 63) / 64 * 64;
  CKI(dalloc(&c->Z, (size_t)m * c->ldz));
  CKI(dalloc(&c->Zt, (size_t)n * c->ldzt));
  if (p->precision == GODEC_PREC_BF16_REFINE) {
    CKI(dalloc(reinterpret_cast<unsigned short**>(&c->Z16), (size_t)m * c->ldz));
    CKI(dalloc(reinterpret_cast<unsigned short**>(&c->Zt16), (size_t)n * c->ldzt));
  }
  if (p->precision == GODEC_PREC_BF16_REFINE || greb || c->naive || c->lingo) {
    const size_t W = 64;   // columns of the correction's [U | A] and [V | B] (2r <= 64)
    CKI(dalloc(&c->RA, (size_t)m * RP));
    CKI(dalloc(&c->RB, (size_t)n * RP));
    CKI(dalloc(&c->Wa, (size_t)m * W));
    CKI(dalloc(&c->Wb, (size_t)n * W));
    CKI(dalloc(&c->Qa, (size_t)m * W));
    CKI(dalloc(&c->Qb, (size_t)n * W));
    CKI(dalloc(&c->Qtmp, (size_t)mx * W));
    CKI(dalloc(&c->Rf, (size_t)8 * W * W));
    CKI(dalloc(&c->cs_ref, (size_t)RP));
    CKI(dalloc(&c->rf_part, (size_t)kRefineParts * W * W));
    CKI(dalloc(&c->rf_g, W * W));
    CKI(dalloc(&c->rf_C, W * W));
    CKI(dalloc(&c->rf_core, W * W));
    CKI(dalloc(&c->rf_U, W * W));
    CKI(dalloc(&c->rf_V, W * W));
    CKI(prepare_refine_kernels());
  }
  CKI(dalloc(&c->A1, (size_t)n * RP));
  CKI(dalloc(&c->A1_orig, (size_t)n * RP));
  // plain GoDec with a given test matrix, on request: its first projection subtracts S A1
  // from a cached X A1 (the other forms change A1 or X between L-steps, or stream a float16
  // copy of Z).  The cost of S A1 grows with k at about the rate of random reads from HBM;
  // at m = n = 10^4 it matches the 94 us product near k = m n / 200 and saves 40 us at
  // k = m n / 1000, but over whole iterations at k = m n / 1000 the lagged normalisers'
  // alarm trips more often with it (8 against 2 in 36 iterations), which costs more than
  // it saves, so streaming stays the default.
  const bool sparse_first = (p->flags & GODEC_FLAG_SPARSE_FIRST) != 0;
  if (A1 && !greb && !c->naive && !c->lingo && !c->Z16 && sparse_first) CKI(dalloc(&c->XA1, (size_t)m * RP));
  CKI(dalloc(&c->P, (size_t)mx * RP));
  CKI(dalloc(&c->Q1, (size_t)m * RP));
  CKI(dalloc(&c->Q2, (size_t)n * RP));
  CKI(dalloc(&c->U, (size_t)m * RP));
  CKI(dalloc(&c->V, (size_t)n * RP));
  CKI(dalloc(&c->sigma, (size_t)RP));
  CKI(dalloc(&c->Um, rr));
  CKI(dalloc(&c->Vm, rr));
  c->RPp = tc_rpp(RP);
  c->ldb = (mx + 7) / 8 * 8;
  CKI(dalloc(reinterpret_cast<unsigned short**>(&c->bt2), (size_t)4 * 2 * RP * c->ldb));
  CKI(cudaMemsetAsync(c->bt2, 0, (size_t)4 * 2 * RP * c->ldb * 2, c->st));
  CKI(dalloc(&c->cs, (size_t)2 * RP));
  CKI(dalloc(&c->rescale_tmp, 2));
  {
    std::vector<float> cs(2 * (size_t)RP, 1.f / kSkinnyScale);
    CKI(cudaMemcpy(c->cs, cs.data(), cs.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  c->tg[0] = tc_geometry(m, n, c->nsm);
  c->tg[1] = tc_geometry(n, m, c->nsm);
  size_t npart = 0;
  for (const TcGeom& g : c->tg) npart = std::max(npart, (size_t)g.tiles * g.maxseg * 128 * RP);
  CKI(dalloc(&c->part, npart));
  c->npart_cap = npart;
  {
    size_t npend = 0;
    for (const TcGeom& g : c->tg) npend = std::max(npend, (size_t)g.G * g.maxpend);
    CKI(dalloc(&c->pend, npend));
    c->npend_cap = npend;
  }
  const int64_t tiles = prod_tiles(mx);
  c->ncounters = tiles;
  CKI(dalloc(&c->counters, (size_t)tiles));
  CKI(cudaMemsetAsync(c->counters, 0, (size_t)tiles * sizeof(unsigned), c->st));
  CKI(dalloc(reinterpret_cast<unsigned short**>(&c->LA), (size_t)m * 128));
  CKI(dalloc(reinterpret_cast<unsigned short**>(&c->LB), (size_t)n * 128));
  {
    const bool ok = make_tmap_f32(c->tmap[5], X, m, n, p->ldx, 128) &&
                    make_tmap_f16(c->tmap[6], c->LA, m, 128, 128, 128) &&
                    make_tmap_f16(c->tmap[7], c->LB, n, 128, 128, 64) &&
                    make_tmap_f32(c->tmap[0], c->Z, m, n, c->ldz, 128) &&
                    make_tmap_f32(c->tmap[1], c->Zt, n, m, c->ldzt, 128) &&
                    make_tmap_f16(c->tmap[2], bt2(c, 0), 2 * RP, m, c->ldb, 2 * RP) &&
                    make_tmap_f16(c->tmap[3], bt2(c, 1), 2 * RP, n, c->ldb, 2 * RP) &&
                    make_tmap_f16(c->tmap[4], bt2(c, 2), 2 * RP, n, c->ldb, 2 * RP);
    const bool ok16 = !c->Z16 ||
                      (make_tmap_f16(c->tmap[8], c->Z16, m, n, c->ldz, 128) &&
                       make_tmap_f16(c->tmap[9], c->Zt16, n, m, c->ldzt, 128));
    const bool ok3 = !(c->Z16 || greb || c->naive || c->lingo) ||
                     (make_tmap_f16(c->tmap[13], bt2(c, 3), 2 * RP, n, c->ldb, 2 * RP) &&
                      make_tmap_f16(c->tmap[14], bt2(c, 3), 2 * RP, m, c->ldb, 2 * RP));
    if (!ok || !ok16 || !ok3) {
      fail(c, GODEC_ERR_CUDA, "tensor map encoding failed");
      return bail(GODEC_ERR_CUDA);
    }
  }
  c->gpart_stride = ((size_t)tiles * rr * sizeof(double) + 255) & ~size_t(255);
  CKI(dalloc(&c->gparts, c->gpart_stride * np));
  CKI(dalloc(&c->g64, (size_t)(np + 2) * rr));
  CKI(dalloc(&c->g32, (size_t)(np + 2) * rr));
  CKI(dalloc(&c->gscr, (size_t)apply_blocks(mx) * rr));
  CKI(dalloc(&c->Rtmp, (size_t)np * 2 * rr));
  CKI(dalloc(&c->Rslot, (size_t)2 * np * rr));
  CKI(dalloc(&c->Tslot, (size_t)2 * np * rr));
  CKI(dalloc(&c->Rfin, 8 * rr));
  CKI(dalloc(&c->Pi, rr));
  CKI(dalloc(&c->Vprev, rr));
  CKI(dalloc(reinterpret_cast<char**>(&c->ctl), sizeof(Ctl)));
  CKI(cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->st));
  const unsigned long long mn = (unsigned long long)(m * n);
  unsigned long long cap = 2ull * (unsigned long long)p->k + 65536ull;
  if (cap > mn) cap = mn;
  if (alloc_candidates(c, cap)) return bail(GODEC_ERR_OOM);
  for (int b = 0; b < 2; ++b) {
    CKI(dalloc(&c->S_idx[b], (size_t)p->k));
    CKI(dalloc(&c->S_val[b], (size_t)p->k));
  }
  c->sbits_words = ((long long)((mn + 31) / 32) + 31) / 32 * 32;   // each bitmap 128-byte aligned
  c->sbits_bytes = 2 * (size_t)c->sbits_words * sizeof(unsigned);
  CKI(dalloc(reinterpret_cast<char**>(&c->sbits), c->sbits_bytes));
  c->idx_bits = 1;
  while ((1ull << c->idx_bits) < mn) ++c->idx_bits;
  launch_fill_zero(c->Q1, (size_t)m * RP * sizeof(float), c->st);
  launch_fill_zero(c->U, (size_t)m * RP * sizeof(float), c->st);
  if (A1) {
    const int a1c = c->naive ? c->np_cols : (c->lingo ? c->lg_d : p->r);
    launch_pad_copy(A1, n, a1c, a1c, c->A1_orig, RP, c->st);
  }
  else launch_fill_zero(c->A1_orig, (size_t)n * RP * sizeof(float), c->st);
  CKI(cudaGetLastError());
  godec_status s = reset_state(c);
  if (s) return bail(s);
  *out = c;
  return GODEC_OK;
#undef CKI
}

godec_status godec_init(godec_ctx** out, const godec_params* p, const float* X, const float* A1,
                        void* stream) {
  if (!out) return GODEC_ERR_ARG;
  *out = nullptr;
  char why[200];
  if (bad_params(p, why, sizeof(why))) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_init: %s", why);
    return GODEC_ERR_ARG;
  }
  if (!X || !A1 || (reinterpret_cast<uintptr_t>(X) & 15)) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_init: X must be a 16-byte aligned device pointer, A1 non-NULL");
    return GODEC_ERR_ARG;
  }
  return init_ctx(out, p, X, A1, stream, false);
}

godec_status godec_reset(godec_ctx* c) {
  if (!c) return GODEC_ERR_ARG;
  return reset_state(c);
}

godec_status godec_iterate(godec_ctx* c, int32_t n_iter, double* rel_err) {
  if (!c) return GODEC_ERR_ARG;
  if (c->greb || c->lingo) return fail(c, GODEC_ERR_STATE, "this context runs through its own entry points");
  if (n_iter < 0) return fail(c, GODEC_ERR_ARG, "n_iter must be >= 0");
  godec_status s = run_iterations(c, n_iter, -1.0);
  if (s) return s;
  if (rel_err) {
    Ctl h;
    if ((s = read_ctl(c, &h))) return s;
    *rel_err = h.rel_err;
  }
  return GODEC_OK;
}

godec_status godec_solve(godec_ctx* c, int32_t* iters, double* rel_err) {
  if (!c) return GODEC_ERR_ARG;
  if (c->greb || c->lingo) return fail(c, GODEC_ERR_STATE, "this context runs through its own entry points");
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  const int remaining = c->p.max_iter - h.iter;
  if (remaining > 0) {
    s = run_iterations(c, remaining, c->p.tol);
    if (s) return s;
  }
  if ((s = read_ctl(c, &h))) return s;
  if (h.converged) {   // leave the context ready for further calls
    launch_reset_iter(c->ctl, c->st);
    CK(cudaStreamSynchronize(c->st));
  }
  if (iters) *iters = h.iter;
  if (rel_err) *rel_err = h.rel_err;
  return GODEC_OK;
}

godec_status godec_check_timeout(godec_ctx* c, uint32_t polls) {
  if (!c) return GODEC_ERR_ARG;
  if (polls < 1 || polls > (1u << 20)) return fail(c, GODEC_ERR_ARG, "polls must be in 1 .. 2^20");
  launch_wait_check(c->ctl, polls, c->st);
  CK(cudaGetLastError());
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  if (h.abort) return handle_abort(c, h);
  return fail(c, GODEC_ERR_STATE, "the self-test wait completed, which nothing should make it do");
}

godec_status godec_profile(godec_ctx* c, int32_t n_iter, double* ms, int64_t* launches,
                           double* bytes_product) {
  if (!c || n_iter < 0) return GODEC_ERR_ARG;
  if (c->greb || c->lingo) return fail(c, GODEC_ERR_STATE, "this context runs through its own entry points");
  if (c->naive || c->lingo) return fail(c, GODEC_ERR_STATE, "godec_profile covers the BRP form only");
  for (int k = 0; k < GODEC_PROF_CLASSES; ++k) {
    if (ms) ms[k] = 0.0;
    if (launches) launches[k] = 0;
  }
  if (bytes_product)
    *bytes_product = 4.0 * (double)c->p.m * (double)c->p.n + 4.0 * (double)(c->p.m + c->p.n) * c->r;
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  const int start = h.iter;
  int guard = 0;
  while (h.iter - start < n_iter) {
    const bool fast = !c->need_exact;
    c->prof = true;
    c->prof_used = 0;
    c->prof_cls.clear();
    c->prof_side.clear();
    enqueue_iteration(c, fast);
    c->prof = false;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    CK(cudaStreamSynchronize(c->side_st));
    CK(cudaStreamSynchronize(c->rank_st));
    for (size_t i = 0; i < c->prof_cls.size(); ++i) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
      const int k = c->prof_cls[i];
      if (ms) ms[k] += t;
      if (launches) launches[k] += 1;
    }
    const int before = h.iter;
    if ((s = read_ctl(c, &h))) return s;
    note_done(c, fast, h.iter - before);
    if (h.abort) {
      if (h.converged) break;
      if ((s = handle_abort(c, h))) return s;
      if (++guard > 64) return fail(c, GODEC_ERR_STATE, "too many aborted iterations");
      if ((s = read_ctl(c, &h))) return s;
    }
  }
  return GODEC_OK;
}

godec_status godec_profile_trace(godec_ctx* c, int32_t cap, int32_t* cls, int32_t* side, float* t0, float* t1,
                                 int32_t* count) {
  if (!c || cap < 0 || !count) return GODEC_ERR_ARG;
  const size_t nl = c->prof_cls.size();
  *count = (int32_t)nl;
  if (nl == 0 || 2 * nl > c->prof_used) return GODEC_OK;
  for (size_t i = 0; i < nl && i < (size_t)cap; ++i) {
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, c->ev_pool[0], c->ev_pool[2 * i]));
    CK(cudaEventElapsedTime(&b, c->ev_pool[0], c->ev_pool[2 * i + 1]));
    if (cls) cls[i] = c->prof_cls[i];
    if (side) side[i] = c->prof_side[i];
    if (t0) t0[i] = a;
    if (t1) t1[i] = b;
  }
  return GODEC_OK;
}

godec_status godec_get_info(godec_ctx* c, godec_info* info) {
  if (!c || !info) return GODEC_ERR_ARG;
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  info->iter = h.iter;
  info->r_eff = c->r;
  info->rel_err = h.rel_err;
  info->obj = h.obj;
  info->normX2 = h.normX2;
  info->nnz = h.nnz_cur;
  info->select_passes = h.last_passes;
  info->rank_drops = c->rank_drops;
  info->launches_per_iter = c->graph_nodes;
  info->exact_iters = c->exact_iters;
  info->svd_sweeps = h.svd_sweeps;
  info->chol_shifts = h.chol_shifts;
  info->alarms = c->alarms;
  return GODEC_OK;
}

godec_status godec_get_L(godec_ctx* c, float* U, float* sigma, float* V, int32_t* r_eff) {
  if (!c) return GODEC_ERR_ARG;
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  if (h.iter == 0) return fail(c, GODEC_ERR_STATE, "no iteration has run yet");
  if (r_eff) *r_eff = c->r;
  if (U) launch_unpad_copy(c->U, c->p.m, c->RP, U, c->r, c->st);
  if (V) launch_unpad_copy(c->V, c->p.n, c->RP, V, c->r, c->st);
  if (sigma) CK(cudaMemcpyAsync(sigma, c->sigma, c->r * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

godec_status godec_get_L_dense(godec_ctx* c, float* L, int64_t ldl) {
  if (!c) return GODEC_ERR_ARG;
  if (!L || ldl < c->p.n) return fail(c, GODEC_ERR_ARG, "godec_get_L_dense: L must be non-NULL with ldl >= n");
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  if (h.iter == 0) return fail(c, GODEC_ERR_STATE, "no iteration has run yet");
  launch_lowrank_dense(c->U, c->RP, c->sigma, c->V, c->RP, c->p.m, c->p.n, c->r, L, ldl, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

godec_status godec_residual(godec_ctx* c, float* R, int64_t ldr) {
  if (!c || !R || ldr < c->p.n) {
    if (c) fail(c, GODEC_ERR_ARG, "godec_residual: R must be non-NULL with ldr >= n");
    return GODEC_ERR_ARG;
  }
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  if (h.iter < 1) return fail(c, GODEC_ERR_STATE, "no iteration has run yet");
  launch_lsplit(c->U, c->V, c->sigma, c->p.m, c->p.n, c->RP, c->r, c->ctl->zscale, c->LA, c->LB, c->st);
  ResidTcLaunch rl{};
  rl.ra.X = c->X;
  rl.ra.m = c->p.m;
  rl.ra.n = c->p.n;
  rl.ra.ctl = c->ctl;
  rl.mapX = c->tmap[5];
  rl.mapA = c->tmap[6];
  rl.mapB = c->tmap[7];
  rl.zscale = c->ctl->zscale;
  rl.dump = R;
  rl.ldd = ldr;
  rl.nsm = c->nsm;
  launch_resid_tc(rl, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

godec_status godec_get_S(godec_ctx* c, int64_t* idx, float* val, int64_t cap, int64_t* nnz) {
  if (!c) return GODEC_ERR_ARG;
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  if (nnz) *nnz = h.nnz_cur;
  if (cap < h.nnz_cur) return fail(c, GODEC_ERR_ARG, "cap %lld < nnz %lld", (long long)cap, h.nnz_cur);
  const long long k = h.nnz_cur;
  if (k == 0) return GODEC_OK;
  if (!idx || !val) return fail(c, GODEC_ERR_ARG, "idx and val must be non-NULL");
  // sort a copy by linear index, in place in the caller's buffers
  size_t scratch = sort_coo_scratch(k);
  void* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, scratch, c->st));
  CK(cudaMemcpyAsync(idx, c->S_idx[h.cur], k * sizeof(long long), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(val, c->S_val[h.cur], k * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
  launch_sort_coo(reinterpret_cast<long long*>(idx), val, k, tmp, scratch, c->idx_bits, c->st);
  CK(cudaGetLastError());
  CK(cudaFreeAsync(tmp, c->st));
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

godec_status godec_run_host(const godec_params* params, const float* X_host, const float* A1_host,
                            int32_t n_iter, void* stream, float* U, float* sigma, float* V,
                            int32_t* r_eff, int64_t* S_idx, float* S_val, int64_t S_cap,
                            int64_t* nnz, int32_t* iters, double* rel_err) {
  char why[200];
  if (bad_params(params, why, sizeof(why)) || !X_host || !A1_host) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_run_host: %s", X_host && A1_host ? why : "NULL input");
    return GODEC_ERR_ARG;
  }
  godec_ctx* c = nullptr;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  godec_params p = *params;
  p.ldx = (p.n + 3) / 4 * 4;
  float *dX = nullptr, *dA = nullptr, *dU = nullptr, *dV = nullptr, *dS = nullptr, *dSv = nullptr;
  long long* dSi = nullptr;
  godec_status s = GODEC_OK;
  int32_t re = 0;
  int64_t cnt = 0;
#define CKH(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      snprintf(g_static_err, sizeof(g_static_err), "godec_run_host: %s: %s", #call,           \
               cudaGetErrorString(e_));                                                       \
      s = e_ == cudaErrorMemoryAllocation ? GODEC_ERR_OOM : GODEC_ERR_CUDA;                   \
      goto done;                                                                              \
    }                                                                                         \
  } while (0)
  CKH(cudaMallocAsync(reinterpret_cast<void**>(&dX), (size_t)p.m * p.ldx * sizeof(float), st));
  CKH(cudaMallocAsync(reinterpret_cast<void**>(&dA), (size_t)p.n * p.r * sizeof(float), st));
  CKH(cudaMemcpy2DAsync(dX, p.ldx * sizeof(float), X_host, p.n * sizeof(float), p.n * sizeof(float),
                        p.m, cudaMemcpyHostToDevice, st));
  CKH(cudaMemcpyAsync(dA, A1_host, (size_t)p.n * p.r * sizeof(float), cudaMemcpyHostToDevice, st));
  s = godec_init(&c, &p, dX, dA, stream);
  if (s) goto done;
  if (n_iter > 0) s = godec_iterate(c, n_iter, rel_err);
  else s = godec_solve(c, iters, rel_err);
  if (s) goto done;
  if (n_iter > 0 && iters) *iters = n_iter;
  CKH(cudaMallocAsync(reinterpret_cast<void**>(&dU), (size_t)p.m * p.r * sizeof(float), st));
  CKH(cudaMallocAsync(reinterpret_cast<void**>(&dV), (size_t)p.n * p.r * sizeof(float), st));
  CKH(cudaMallocAsync(reinterpret_cast<void**>(&dS), (size_t)p.r * sizeof(float), st));
  s = godec_get_L(c, dU, dS, dV, &re);
  if (s) goto done;
  if (r_eff) *r_eff = re;
  if (U) CKH(cudaMemcpyAsync(U, dU, (size_t)p.m * re * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (V) CKH(cudaMemcpyAsync(V, dV, (size_t)p.n * re * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (sigma) CKH(cudaMemcpyAsync(sigma, dS, (size_t)re * sizeof(float), cudaMemcpyDeviceToHost, st));
  {
    godec_info info;
    s = godec_get_info(c, &info);
    if (s) goto done;
    cnt = info.nnz;
  }
  if (nnz) *nnz = cnt;
  if (S_idx && S_val && cnt > 0) {
    if (S_cap < cnt) { s = GODEC_ERR_ARG; snprintf(g_static_err, sizeof(g_static_err), "godec_run_host: S_cap < nnz"); goto done; }
    CKH(cudaMallocAsync(reinterpret_cast<void**>(&dSi), (size_t)cnt * sizeof(long long), st));
    CKH(cudaMallocAsync(reinterpret_cast<void**>(&dSv), (size_t)cnt * sizeof(float), st));
    s = godec_get_S(c, reinterpret_cast<int64_t*>(dSi), dSv, cnt, &cnt);
    if (s) goto done;
    CKH(cudaMemcpyAsync(S_idx, dSi, (size_t)cnt * sizeof(long long), cudaMemcpyDeviceToHost, st));
    CKH(cudaMemcpyAsync(S_val, dSv, (size_t)cnt * sizeof(float), cudaMemcpyDeviceToHost, st));
  }
  CKH(cudaStreamSynchronize(st));
done:
  if (s && c) snprintf(g_static_err, sizeof(g_static_err), "godec_run_host: %.200s", c->err);
  godec_destroy(c);
  void* ptrs[] = {dX, dA, dU, dV, dS, dSi, dSv};
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, st);
  cudaStreamSynchronize(st);
  return s;
#undef CKH
}

godec_status godec_hard_threshold(const float* R, int64_t m, int64_t n, int64_t ldr, int64_t k,
                                  int64_t* idx, float* val, int64_t cap, int64_t* nnz, void* stream) {
  // A context with r = 0 (L = 0) and no working copy of X - S: only the S-step runs.
  if (!R || m < 1 || n < 1 || ldr < n || (ldr * 4) % 16 || k < 0 || k > m * n ||
      (double)m * (double)n >= 4294967296.0 || (reinterpret_cast<uintptr_t>(R) & 15)) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_hard_threshold: invalid argument");
    return GODEC_ERR_ARG;
  }
  godec_ctx* c = new (std::nothrow) godec_ctx;
  if (!c) return GODEC_ERR_OOM;
  godec_status s = GODEC_OK;
  c->st = reinterpret_cast<cudaStream_t>(stream);
  c->p.m = m;
  c->p.n = n;
  c->p.ldx = ldr;
  c->p.k = k;
  c->p.r = 0;
  c->RP = 8;
  c->X = R;
  do {
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess ||
        prepare_select_kernels() != cudaSuccess) {
      s = fail(c, GODEC_ERR_CUDA, "no CUDA device");
      break;
    }
    const unsigned long long mn = (unsigned long long)(m * n);
    unsigned long long cap0 = 2ull * (unsigned long long)k + 65536ull;
    if (cap0 > mn) cap0 = mn;
    if (dalloc(&c->ctl, 1) != cudaSuccess || dalloc(&c->U, (size_t)m * 8) != cudaSuccess ||
        dalloc(&c->V, (size_t)n * 8) != cudaSuccess || dalloc(&c->sigma, 8) != cudaSuccess ||
        dalloc(&c->S_idx[0], (size_t)k) != cudaSuccess || dalloc(&c->S_idx[1], (size_t)k) != cudaSuccess ||
        dalloc(&c->S_val[0], (size_t)k) != cudaSuccess || dalloc(&c->S_val[1], (size_t)k) != cudaSuccess) {
      s = fail(c, GODEC_ERR_OOM, "out of device memory");
      break;
    }
    if ((s = alloc_candidates(c, cap0))) break;
    c->idx_bits = 1;
    while ((1ull << c->idx_bits) < mn) ++c->idx_bits;
    if (cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->st) != cudaSuccess) {
      s = fail(c, GODEC_ERR_CUDA, "memset");
      break;
    }
    Ctl h;
    memset(&h, 0, offsetof(Ctl, hist));
    h.k_req = k;
    h.k_eff = k;
    h.tol = -1.0;
    h.normX2 = 1.0;
    cudaMemcpyAsync(c->ctl, &h, offsetof(Ctl, hist), cudaMemcpyHostToDevice, c->st);
    launch_reset_iter(c->ctl, c->st);
    for (int attempt = 0; attempt < 8; ++attempt) {
      enqueue_sstep(c, 0);
      Ctl hh;
      if ((s = read_ctl(c, &hh))) break;
      if (hh.nonfinite) { s = fail(c, GODEC_ERR_NONFINITE, "non-finite values in R"); break; }
      if (!hh.abort) break;
      if (!hh.need_bigger_cand) { s = fail(c, GODEC_ERR_STATE, "selection aborted"); break; }
      unsigned long long cap2 = std::min<unsigned long long>(c->cap * 2, mn);
      if ((s = alloc_candidates(c, cap2))) break;
      launch_reset_iter(c->ctl, c->st);
    }
    if (s) break;
    s = godec_get_S(c, idx, val, cap, nnz);
  } while (0);
  if (s) snprintf(g_static_err, sizeof(g_static_err), "godec_hard_threshold: %.200s", c->err);
  godec_destroy(c);
  return s;
}

// ---- streaming primitives ----------------------------------------------------------------
static godec_status mul_common(const float* Z, int64_t m, int64_t n, int64_t ldz, const float* B, int32_t r,
                               float* Y, void* stream, int trans) {
  if (!Z || !B || !Y || m < 1 || n < 1 || ldz < n || (ldz * 4) % 16 || r < 1 || r > GODEC_MAX_RANK ||
      (reinterpret_cast<uintptr_t>(Z) & 15)) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: invalid argument");
    return GODEC_ERR_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int RP = round_up(r, 8);
  const int64_t rows = trans ? n : m, K = trans ? m : n;
  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      prepare_tc_kernels() != cudaSuccess) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: no CUDA device");
    return GODEC_ERR_CUDA;
  }
  const TcGeom geom = tc_geometry(rows, K, nsm);
  const int64_t ldt = (m + 3) / 4 * 4, ldb = (K + 7) / 8 * 8;
  float *Bp = nullptr, *part = nullptr, *Yp = nullptr, *Zt = nullptr, *aux = nullptr;
  void* Bs = nullptr;
  unsigned* cnt = nullptr;
  int* pend = nullptr;
  bool ok = cudaMallocAsync(reinterpret_cast<void**>(&Bp), (size_t)K * RP * sizeof(float), st) == cudaSuccess &&
            cudaMallocAsync(&Bs, (size_t)2 * RP * ldb * 2, st) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&aux), (size_t)(4 + RP) * sizeof(float), st) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&part), (size_t)geom.tiles * geom.maxseg * 128 * RP * sizeof(float),
                            st) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&Yp), (size_t)rows * RP * sizeof(float), st) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&cnt), (size_t)geom.tiles * sizeof(unsigned), st) == cudaSuccess &&
            cudaMallocAsync(reinterpret_cast<void**>(&pend), (size_t)geom.G * geom.maxpend * sizeof(int), st) ==
                cudaSuccess &&
            (!trans || cudaMallocAsync(reinterpret_cast<void**>(&Zt), (size_t)n * ldt * sizeof(float), st) == cudaSuccess);
  bool mapped = false;
  if (ok) {
    alignas(64) unsigned char mapA[128], mapB[128];
    mapped = make_tmap_f32(mapA, trans ? Zt : Z, rows, K, trans ? ldt : ldz, 128) &&
             make_tmap_f16(mapB, Bs, 2 * RP, K, ldb, 2 * RP);
    if (mapped && cudaMemsetAsync(cnt, 0, (size_t)geom.tiles * sizeof(unsigned), st) != cudaSuccess) {
      for (void* q : {(void*)Bp, Bs, (void*)aux, (void*)part, (void*)Yp, (void*)cnt, (void*)pend, (void*)Zt})
        if (q) cudaFreeAsync(q, st);
      snprintf(g_static_err, sizeof(g_static_err), "godec_mul: clearing the tile counters: %s",
               cudaGetErrorString(cudaGetLastError()));
      return GODEC_ERR_CUDA;
    }
    if (mapped) {
      // aux: {s_Z, 1/s_Z}, max-|Z| scratch, pad, then RP column factors of B
      launch_zscale(Z, m, n, ldz, reinterpret_cast<unsigned*>(aux + 2), aux, nsm, st);
      launch_pad_copy(B, K, r, r, Bp, RP, st);
      launch_split_t(Bp, K, RP, Bs, ldb, aux + 4, st);
      if (trans) launch_transpose(Z, m, n, ldz, Zt, ldt, st);
      TcLaunch l{};
      l.mapA = mapA;
      l.mapB = mapB;
      l.rows = rows;
      l.K = K;
      l.RP = RP;
      l.geom = geom;
      l.part = part;
      l.counters = cnt;
      l.out = Yp;
      l.cscale = aux + 4;
      l.zscale = aux;
      l.pend = pend;
      launch_prod_tc(l, st);
      launch_unpad_copy(Yp, rows, RP, Y, r, st);
    }
  }
  void* ptrs[] = {Bp, Bs, aux, part, Yp, cnt, pend, Zt};
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, st);
  if (!ok) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: out of device memory");
    return GODEC_ERR_OOM;
  }
  if (!mapped) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: tensor map encoding failed");
    return GODEC_ERR_CUDA;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  return GODEC_OK;
}

godec_status godec_mul_ZB(const float* Z, int64_t m, int64_t n, int64_t ldz, const float* B, int32_t r,
                          float* Y, void* stream) {
  return mul_common(Z, m, n, ldz, B, r, Y, stream, 0);
}

godec_status godec_mul_ZtC(const float* Z, int64_t m, int64_t n, int64_t ldz, const float* C, int32_t r,
                           float* W, void* stream) {
  return mul_common(Z, m, n, ldz, C, r, W, stream, 1);
}

// ---- GreBsmo (Sec. 3.2.1, Algorithm 2) --------------------------------------------------
// The context's buffers take these roles: V holds the unit-column V^T (n x RP) that the
// next product reads, Q1 the orthonormal U (m x RP), Q2 W = Z^T U (n x RP, so that
// L = U W^T), sigma the column norms of W; A1, Qa, Qb, P are work space of the increments.
// Columns at and beyond the current rank are zero everywhere.

// The random-projection increment: `add` new unit rows of V (columns ri .. ri+add-1 of
// c->V), the top right singular vectors of D from test matrix Omega_stage.
static void greb_increment(godec_ctx* c, int ri, int add, int stage) {
  const int RP = c->RP, p = c->gp.dr + c->gp.oversample;
  const int64_t m = c->p.m, n = c->p.n;
  cudaStream_t st = c->st;
  const size_t q = (size_t)64 * 64;
  float *R1 = c->Rf, *T1 = R1 + q, *R2m = T1 + q, *T2 = R2m + q;
  launch_fill_zero(c->A1, (size_t)n * RP * sizeof(float), st);
  launch_pad_copy(c->omega + (size_t)stage * n * p, n, p, p, c->A1, RP, st);
  cqr2(c, c->A1, n, p, RP, c->Qb, R1, T1, R2m, T2);                 // B = orth(Omega)
  for (int s = 0; s < c->gp.q_inc; ++s) {
    greb_apply_D(c, ri, p, c->Qb, c->P);
    cqr2(c, c->P, m, p, RP, c->Qa, R1, T1, R2m, T2);                // orth(D B)
    greb_apply_Dt(c, ri, p, c->Qa, c->P);
    cqr2(c, c->P, n, p, RP, c->Qb, R1, T1, R2m, T2);                // B = orth(D^T orth(D B))
  }
  greb_apply_D(c, ri, p, c->Qb, c->P);                               // Y = D B = Qa R2m R1
  cqr2(c, c->P, m, p, RP, c->Qa, R1, T1, R2m, T2);
  launch_rmul(R2m, R1, RP, p, c->rf_core, 0, nullptr, st);
  launch_svd_small(c->rf_core, p, add, c->rf_U, c->cs_ref + 0, c->rf_V, st, nullptr, true);   // right vectors of Y
  launch_tall_small_d(c->Qb, RP, p, c->rf_V, add, 0, add, n, 1.f, 0.f, c->V + ri, RP, st);
}

// The factor updates of one inner step of eq. GreBsmoA at rank ri: U = orth(Z V^T),
// W = Z^T U (V = W^T), kept as sigma (column norms of W) and its unit columns.
static void greb_lstep(godec_ctx* c, int ri) {
  const int RP = c->RP;
  const int64_t m = c->p.m, n = c->p.n;
  const size_t rr = (size_t)RP * RP;
  cudaStream_t st = c->st;
  launch_split_t(c->V, n, RP, bt2(c, 2), c->ldb, c->cs, st);
  greb_prod(c, true, 4, c->cs, c->P, 1, 0);
  gram_sum(c, gpart(c, 0), 0, prod_tiles(m), g64(c, 0), st);
  final_cqr2(c, m, g64(c, 0), c->Rfin, c->Rfin + 2 * rr, c->Q1, g64(c, 2), bt2(c, 0));
  greb_prod(c, false, 2, c->cs + RP, c->Q2, 1, 1);
  gram_sum(c, gpart(c, 1), 0, prod_tiles(n), g64(c, 1), st);
  launch_colnorm(c->Q2, g64(c, 1), n, RP, ri, c->V, c->sigma, c->nsm, st);
}

// The S-step of the inner step: S = S_lambda(X - U W^T) (eq. softt) and the sparse update
// of Z = X - S.  L = U diag(sigma) V^T with V the unit columns of W.
static void greb_sstep(godec_ctx* c, int ri, unsigned guess, const float* U, float lambda) {
  const int RP = c->RP;
  const int64_t m = c->p.m, n = c->p.n;
  cudaStream_t st = c->st;
  launch_reset_iter(c->ctl, st);
  launch_soft_plan(c->ctl, guess, st);
  launch_lsplit(U, c->V, c->sigma, m, n, RP, ri, c->ctl->zscale, c->LA, c->LB, st);
  ResidTcLaunch rl{};
  rl.ra.X = c->X;
  rl.ra.m = m;
  rl.ra.n = n;
  rl.ra.ldx = c->p.ldx;
  rl.ra.r = ri;
  rl.ra.RP = RP;
  rl.ra.pass = 0;
  rl.ra.ctl = c->ctl;
  rl.ra.cand_key = c->cand_key;
  rl.ra.cand_idx = c->cand_idx;
  rl.ra.cand_val = c->cand_val;
  rl.ra.cand_cap = c->cap;
  rl.mapX = c->tmap[5];
  rl.mapA = c->tmap[6];
  rl.mapB = c->tmap[7];
  rl.zscale = c->ctl->zscale;
  rl.nsm = c->nsm;
  launch_resid_tc(rl, st);
  SoftEmitArgs se{};
  se.ctl = c->ctl;
  se.cand_idx = c->cand_idx;
  se.cand_val = c->cand_val;
  se.cand_cap = c->cap;
  se.s_cap = c->p.k;
  for (int b = 0; b < 2; ++b) {
    se.S_idx[b] = c->S_idx[b];
    se.S_val[b] = c->S_val[b];
  }
  se.sbits = c->sbits;
  se.sbits_words = c->sbits_words;
  se.lambda = lambda;
  launch_emit_soft(se, c->nsm, st);
  EmitArgs ea{};
  ea.ctl = c->ctl;
  ea.S_idx[0] = c->S_idx[0];
  ea.S_idx[1] = c->S_idx[1];
  ea.S_val[0] = c->S_val[0];
  ea.S_val[1] = c->S_val[1];
  ea.X = c->X;
  ea.n = n;
  ea.ldx = c->p.ldx;
  ea.Z = c->Z;
  ea.ldz = c->ldz;
  ea.Zt = c->Zt;
  ea.ldzt = c->ldzt;
  ea.zscale = c->ctl->zscale;
  ea.max_nnz = c->p.k;
  ea.sbits = c->sbits;
  ea.sbits_words = c->sbits_words;
  launch_z_update(ea, c->nsm, st);
}

// Grow the S and candidate buffers to hold `need` entries (keeping the committed S).
static godec_status greb_grow(godec_ctx* c, const Ctl& h, unsigned long long need) {
  unsigned long long cap = std::max<unsigned long long>(2 * c->cap, need + 65536ull);
  const unsigned long long mn = (unsigned long long)(c->p.m * c->p.n);
  if (cap > mn) cap = mn;
  if (godec_status s = alloc_candidates(c, cap)) return s;
  const long long k = (long long)std::min<unsigned long long>(mn, std::max<unsigned long long>(2 * (unsigned long long)c->p.k, need + 65536ull));
  for (int b = 0; b < 2; ++b) {
    long long* ni = nullptr;
    float* nv = nullptr;
    CK(dalloc(&ni, (size_t)k));
    CK(dalloc(&nv, (size_t)k));
    if (b == h.cur && h.nnz_cur > 0) {
      CK(cudaMemcpyAsync(ni, c->S_idx[b], (size_t)h.nnz_cur * sizeof(long long), cudaMemcpyDeviceToDevice, c->st));
      CK(cudaMemcpyAsync(nv, c->S_val[b], (size_t)h.nnz_cur * sizeof(float), cudaMemcpyDeviceToDevice, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    cudaFree(c->S_idx[b]);
    cudaFree(c->S_val[b]);
    c->S_idx[b] = ni;
    c->S_val[b] = nv;
  }
  c->p.k = k;
  return GODEC_OK;
}

int godec_naive_columns(int64_t m, int64_t n, int32_t r) {
  int64_t p = (int64_t)r + 8;
  p = std::min<int64_t>(p, GODEC_MAX_RANK);
  p = std::min<int64_t>(p, std::min(m, n));
  return (int)std::max<int64_t>(p, r);
}

godec_status godec_naive_init(godec_ctx** out, const godec_params* p, const float* X, const float* Omega,
                              void* stream) {
  if (!out) return GODEC_ERR_ARG;
  *out = nullptr;
  char why[200];
  if (bad_params(p, why, sizeof(why))) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_naive_init: %s", why);
    return GODEC_ERR_ARG;
  }
  if (p->precision != GODEC_PREC_FP32 || p->q < 1) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_naive_init: needs precision GODEC_PREC_FP32 and q >= 1");
    return GODEC_ERR_ARG;
  }
  if (!X || !Omega || (reinterpret_cast<uintptr_t>(X) & 15)) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_naive_init: X must be a 16-byte aligned device pointer, Omega non-NULL");
    return GODEC_ERR_ARG;
  }
  return init_ctx(out, p, X, Omega, stream, false, godec_naive_columns(p->m, p->n, p->r));
}

godec_status godec_grebsmo_init(godec_ctx** out, const godec_grebsmo_params* gp, const float* X,
                                const float* Omega, void* stream) {
  if (!out) return GODEC_ERR_ARG;
  *out = nullptr;
  const char* why = nullptr;
  if (!gp) why = "params is NULL";
  else if (gp->m < 1 || gp->n < 1 || (double)gp->m * (double)gp->n >= 4294967296.0) why = "need m, n >= 1, m*n < 2^32";
  else if (gp->ldx < gp->n || (gp->ldx * 4) % 16) why = "ldx must be >= n and ldx*4 a multiple of 16";
  else if (!(gp->lambda > 0.0) || !std::isfinite(gp->lambda)) why = "lambda must be finite and > 0";
  else if (gp->dr < 1 || gp->K < 1) why = "dr and K must be >= 1";
  else if (gp->r_max < gp->dr || gp->r_max > GODEC_MAX_RANK || gp->r_max > gp->m || gp->r_max > gp->n)
    why = "need dr <= r_max <= min(m, n, GODEC_MAX_RANK)";
  else if (gp->oversample < 0 || gp->dr + gp->oversample > GODEC_MAX_RANK || gp->dr + gp->oversample > gp->m ||
           gp->dr + gp->oversample > gp->n)
    why = "need dr + oversample <= min(m, n, GODEC_MAX_RANK)";
  else if (gp->q_inc < 0 || gp->q_inc > 16) why = "q_inc must be in [0, 16]";
  else if (gp->s_cap < 0) why = "s_cap must be >= 0";
  else if (gp->flags & ~GODEC_FLAG_FP64_FACTOR) why = "unknown flags";
  else if (!X || !Omega || (reinterpret_cast<uintptr_t>(X) & 15)) why = "X (16-byte aligned) and Omega must be device pointers";
  if (why) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_grebsmo_init: %s", why);
    return GODEC_ERR_ARG;
  }
  godec_params p{};
  p.m = gp->m;
  p.n = gp->n;
  p.ldx = gp->ldx;
  p.r = std::max(gp->r_max, gp->dr + gp->oversample);
  p.q = 0;
  p.k = std::min<int64_t>(std::max<int64_t>(gp->s_cap, 1), gp->m * gp->n);
  p.tol = -1.0;
  p.max_iter = 1;
  p.precision = GODEC_PREC_FP32;
  p.flags = gp->flags;
  godec_status s = init_ctx(out, &p, X, nullptr, stream, true);
  if (s) return s;
  (*out)->gp = *gp;
  (*out)->omega = Omega;
  return GODEC_OK;
}

// ---- LinGoDec (Sec. 4.3, eqs. LinGoDec and NLinGoDec) -----------------------------------
// W-step (readings R20, R21): with F = Qf Rf (fixed), Y = X - S:  Y Qf = Qy Ry (CholeskyQR2 of
// the streamed product), Ry = Ur S Vr^T (float64), W = Qy Ur S Vr^T Rf^{-T}; then
// L = W F^T = (Qy Ur) S (Qf Vr)^T, kept as U = Qy Ur, V = Qf Vr.  S-step: S_lambda(X - L).
static void lingo_lstep(godec_ctx* c) {
  const int RP = c->RP, d = c->lg_d, r = c->p.r;
  const int64_t m = c->p.m, n = c->p.n;
  const size_t rr = (size_t)RP * RP;
  cudaStream_t st = c->st;
  const int* ab = &c->ctl->abort;
  greb_prod(c, true, 4, c->cs, c->P, 1, 0);                        // Y Qf (operand set at reset)
  gram_sum(c, gpart(c, 0), 0, prod_tiles(m), g64(c, 0), st);
  c->r = d;
  final_cqr2(c, m, g64(c, 0), c->Rfin, c->Rfin + 2 * rr, c->Q1, g64(c, 2), nullptr);   // Y Qf = Qy Rb Ra
  c->r = r;
  launch_rmul(c->Rfin + 2 * rr, c->Rfin, RP, d, c->rf_core, 0, nullptr, st, ab);
  launch_svd_small(c->rf_core, d, r, c->rf_U, c->sigma, c->rf_V, st, ab, true);
  launch_tall_small_d(c->Q1, RP, d, c->rf_U, r, 0, r, m, 1.f, 0.f, c->U, RP, st, ab);
  launch_tall_small_d(c->Q2, RP, d, c->rf_V, r, 0, r, n, 1.f, 0.f, c->V, RP, st, ab);
}

godec_status godec_lingodec_init(godec_ctx** out, const godec_params* p, double lambda, const float* X, const float* F,
                                 int32_t d, void* stream) {
  if (!out) return GODEC_ERR_ARG;
  *out = nullptr;
  char why[200];
  if (bad_params(p, why, sizeof(why))) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_lingodec_init: %s", why);
    return GODEC_ERR_ARG;
  }
  if (p->precision != GODEC_PREC_FP32 || d < 1 || d > GODEC_MAX_RANK || d > p->n || p->r > d ||
      !(lambda > 0.0) || !std::isfinite(lambda) || !X || !F || (reinterpret_cast<uintptr_t>(X) & 15)) {
    snprintf(g_static_err, sizeof(g_static_err),
             "godec_lingodec_init: needs precision FP32, 1 <= r <= d <= min(n, %d), lambda > 0, X (16-byte "
             "aligned) and F device pointers", GODEC_MAX_RANK);
    return GODEC_ERR_ARG;
  }
  godec_params q = *p;
  q.k = std::min<int64_t>(std::max<int64_t>(p->k, 1), p->m * p->n);
  return init_ctx(out, &q, X, F, stream, false, 0, d, lambda);
}

godec_status godec_lingodec_iterate(godec_ctx* c, int32_t n_iter, double* rel_err) {
  if (!c || !c->lingo) {
    if (c) fail(c, GODEC_ERR_STATE, "godec_lingodec_iterate needs a context from godec_lingodec_init");
    return c ? GODEC_ERR_STATE : GODEC_ERR_ARG;
  }
  if (n_iter < 0) return fail(c, GODEC_ERR_ARG, "n_iter must be >= 0");
  const float lamf = (float)c->lg_lambda;
  unsigned guess;
  memcpy(&guess, &lamf, sizeof(guess));
  guess += 1u;   // S is nonzero where |R| > lambda
  godec_status s;
  for (int it = 0; it < n_iter; ++it) {
    lingo_lstep(c);
    for (int attempt = 0;; ++attempt) {
      greb_sstep(c, c->p.r, guess, c->U, (float)c->lg_lambda);
      CK(cudaGetLastError());
      Ctl h;
      if ((s = read_ctl(c, &h))) return s;
      if (h.timeout) return fail(c, GODEC_ERR_TIMEOUT, "a device-side wait of the tensor-core product timed out");
      if (h.nonfinite) return fail(c, GODEC_ERR_NONFINITE, "non-finite values in X - W F^T");
      if (h.abort && h.need_bigger_cand && attempt < 8) {
        if ((s = clear_counters(c))) return s;
        if ((s = rebuild_sbits(c))) return s;
        if ((s = greb_grow(c, h, h.cand_count))) return s;
        continue;
      }
      if (h.abort) return fail(c, GODEC_ERR_STATE, "LinGoDec iteration aborted");
      if (h.range_err) {
        if ((s = rescale_z(c))) return s;
        if ((s = SET_CTL(range_err, 0))) return s;
      }
      if (rel_err) *rel_err = h.rel_err;
      break;
    }
  }
  return GODEC_OK;
}

godec_status godec_lingodec_get_W(godec_ctx* c, float* W) {
  if (!c || !c->lingo || !W) {
    if (c) fail(c, GODEC_ERR_ARG, "godec_lingodec_get_W needs a LinGoDec context and W");
    return GODEC_ERR_ARG;
  }
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  if (h.iter == 0) return fail(c, GODEC_ERR_STATE, "no iteration has run yet");
  const size_t q = (size_t)64 * 64;
  const float *T1 = c->Rf + q, *T2 = c->Rf + 3 * q;
  launch_lingo_g(T1, T2, c->RP, c->rf_V, c->sigma, c->lg_d, c->p.r, c->rf_C, c->st);
  launch_tall_small_d(c->U, c->RP, c->p.r, c->rf_C, c->p.r, 1, c->lg_d, c->p.m, 1.f, 0.f, W, c->lg_d, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

// ---- MSE training (Sec. 4.2.1, Algorithm 4) ----------------------------------------------
// One q = 0 BRP L-step of Algorithm 1 on the context's (re-gathered) matrix with test matrix
// A1 (first r columns, row stride lda): refresh the working copies, set A1, run the L-step
// eagerly (no S-step, no graph), leave the factors in U, sigma, V.
static godec_status mse_block_brp(godec_ctx* c, const float* A1, int lda) {
  cudaStream_t st = c->st;
  const int64_t m = c->p.m, n = c->p.n;
  launch_reset_iter(c->ctl, st);
  launch_zscale(c->X, m, n, c->p.ldx, &c->ctl->zmax_bits, c->ctl->zscale, c->nsm, st);
  launch_scale_copy(c->X, m, n, c->p.ldx, c->Z, c->ldz, c->ctl->zscale, c->nsm, st);
  launch_transpose(c->X, m, n, c->p.ldx, c->Zt, c->ldzt, st, c->ctl->zscale);
  launch_fill_zero(c->A1, (size_t)n * c->RP * sizeof(float), st);
  launch_pad_copy(A1, n, c->p.r, lda, c->A1, c->RP, st);
  launch_split_t(c->A1, n, c->RP, bt2(c, 2), c->ldb, c->cs, st);
  c->r = c->p.r;
  enqueue_lstep(c, false);
  Ctl h;
  if (godec_status s = read_ctl(c, &h)) return s;
  if (h.abort) return fail(c, GODEC_ERR_STATE, "block L-step abandoned (rank %s%s)", h.rank_drop ? "drop" : "ok",
                           h.nonfinite ? ", non-finite values" : "");
  return GODEC_OK;
}

// Block coordinate descent over the label blocks L^1 .. L^k and S, with R = X - sum L^i - S
// kept densely.  Block i: N = R[Omega_i] + L^i[Omega_i] gathered into its own buffer, whose
// GoDec context (q = 0) gives the q = 0 BRP of Algorithm 4 with the test matrix of this step
// (one iteration from S = 0: its L-step is the BRP of N; its S-step is not used); then
// R[Omega_i] = N - L^i_new.  S-step: the top-K of X - sum L^i = R + S_old.
godec_status godec_mse_train(const float* X, int64_t n, int64_t p, int64_t ldx, const int32_t* labels, int32_t k,
                             const int32_t* ranks, int64_t K, int32_t iters, const float* A1s, int32_t r_stride,
                             float* C, float* Lsum, int64_t ldl, int64_t* S_idx, float* S_val, int64_t S_cap,
                             int64_t* nnz, double* history, void* stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const char* why = nullptr;
  if (!X || !labels || !ranks || !A1s || n < 1 || p < 1 || ldx < p || (ldx * 4) % 16 || k < 1 || iters < 1 ||
      K < 0 || K > n * p || r_stride < 1 || r_stride > GODEC_MAX_RANK || (double)n * (double)p >= 4294967296.0 ||
      (reinterpret_cast<uintptr_t>(X) & 15) || (Lsum && ldl < p))
    why = "invalid argument";
  std::vector<std::vector<int64_t>> rows(k > 0 ? k : 0);
  std::vector<float> invD(n > 0 ? n : 0, 0.f);
  if (!why) {
    for (int64_t i = 0; i < n; ++i) {
      int d = 0;
      for (int j = 0; j < k; ++j)
        if (labels[i * k + j]) {
          rows[j].push_back(i);
          ++d;
        }
      invD[i] = d > 0 ? 1.f / (float)d : 0.f;
    }
    for (int j = 0; j < k && !why; ++j)
      if (ranks[j] < 1 || ranks[j] > r_stride || (int64_t)ranks[j] > std::min<int64_t>((int64_t)rows[j].size(), p))
        why = "every rank must satisfy 1 <= r_i <= min(|Omega_i|, p, r_stride)";
  }
  if (why) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mse_train: %s", why);
    return GODEC_ERR_ARG;
  }
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mse_train: no CUDA device");
    return GODEC_ERR_CUDA;
  }
  const int64_t ldr = (p + 3) / 4 * 4;
  std::vector<void*> owned;
  std::vector<godec_ctx*> ctx(k, nullptr);
  godec_status status = GODEC_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (godec_ctx* c : ctx) godec_destroy(c);
    for (void* q : owned) cudaFree(q);
  };
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes ? bytes : 16) != cudaSuccess) return false;
    owned.push_back(*ptr);
    return true;
  };
#define MSE_FAIL(code, ...)                                                  \
  do {                                                                       \
    snprintf(g_static_err, sizeof(g_static_err), "godec_mse_train: " __VA_ARGS__); \
    cleanup();                                                               \
    return code;                                                             \
  } while (0)
  float *R = nullptr, *dinvD = nullptr, *Sv[2] = {nullptr, nullptr};
  int64_t* Si[2] = {nullptr, nullptr};
  double* dsum = nullptr;
  if (!alloc((void**)&R, (size_t)n * ldr * 4) || !alloc((void**)&dinvD, (size_t)n * 4) ||
      !alloc((void**)&dsum, 8) || !alloc((void**)&Si[0], (size_t)std::max<int64_t>(K, 1) * 8) ||
      !alloc((void**)&Sv[0], (size_t)std::max<int64_t>(K, 1) * 4))
    MSE_FAIL(GODEC_ERR_OOM, "out of device memory");
  std::vector<int64_t*> drows(k, nullptr);
  std::vector<float*> N(k, nullptr), U(k, nullptr), sg(k, nullptr), V(k, nullptr);
  for (int j = 0; j < k; ++j) {
    const int64_t nr = (int64_t)rows[j].size();
    if (!alloc((void**)&drows[j], (size_t)nr * 8) || !alloc((void**)&N[j], (size_t)nr * ldr * 4) ||
        !alloc((void**)&U[j], (size_t)nr * ranks[j] * 4) || !alloc((void**)&sg[j], (size_t)ranks[j] * 4) ||
        !alloc((void**)&V[j], (size_t)p * ranks[j] * 4))
      MSE_FAIL(GODEC_ERR_OOM, "out of device memory");
    if (cudaMemcpyAsync(drows[j], rows[j].data(), (size_t)nr * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(N[j], 0, (size_t)nr * ldr * 4, st) != cudaSuccess)
      MSE_FAIL(GODEC_ERR_CUDA, "copy of the label rows failed");
  }
  if (cudaMemcpyAsync(dinvD, invD.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
    MSE_FAIL(GODEC_ERR_CUDA, "copy failed");
  // one context per block, over its gathered rows
  for (int j = 0; j < k; ++j) {
    godec_params q{};
    q.m = (int64_t)rows[j].size();
    q.n = p;
    q.ldx = ldr;
    q.r = ranks[j];
    q.q = 0;
    q.k = 1;
    q.tol = -1.0;
    q.max_iter = 1 << 30;
    q.precision = GODEC_PREC_FP32;
    if ((status = init_ctx(&ctx[j], &q, N[j], nullptr, stream, false))) {
      char why2[200];
      snprintf(why2, sizeof(why2), "%s", g_static_err);
      MSE_FAIL(status, "block %d: %s", j, why2);
    }
  }
  launch_mse_init(X, ldx, dinvD, n, p, R, ldr, nsm, st);
  int64_t nnz_cur = 0;
  std::vector<int> r_eff(ranks, ranks + k);
  for (int t = 0; t < iters; ++t) {
    for (int j = 0; j < k; ++j) {
      godec_ctx* c = ctx[j];
      const int64_t nr = (int64_t)rows[j].size();
      launch_mse_gather(R, ldr, drows[j], nr, p, X, ldx, dinvD, t == 0 ? nullptr : U[j], r_eff[j], sg[j], V[j],
                        r_eff[j], r_eff[j], N[j], ldr, nsm, st);
      if ((status = mse_block_brp(c, A1s + ((size_t)t * k + j) * p * r_stride, r_stride)))
        MSE_FAIL(status, "block %d: %s", j, c->err);
      const int re = c->r;
      launch_unpad_copy(c->U, c->p.m, c->RP, U[j], re, st);
      launch_unpad_copy(c->V, c->p.n, c->RP, V[j], re, st);
      cudaMemcpyAsync(sg[j], c->sigma, (size_t)re * sizeof(float), cudaMemcpyDeviceToDevice, st);
      r_eff[j] = re;
      launch_mse_scatter(R, ldr, drows[j], nr, p, N[j], ldr, U[j], re, sg[j], V[j], re, re, nsm, st);
    }
    // S-step on X - sum L^i = R + S_old
    launch_sparse_axpy(R, ldr, p, Si[0], Sv[0], nnz_cur, 1.f, nsm, st);
    int64_t got = 0;
    godec_status hs = godec_hard_threshold(R, n, p, ldr, K, Si[0], Sv[0], std::max<int64_t>(K, 1), &got, stream);
    if (hs) {
      char why2[200];
      snprintf(why2, sizeof(why2), "%s", g_static_err);
      MSE_FAIL(hs, "S-step: %s", why2);
    }
    nnz_cur = got;
    launch_sparse_axpy(R, ldr, p, Si[0], Sv[0], nnz_cur, -1.f, nsm, st);
    cudaMemsetAsync(dsum, 0, sizeof(double), st);   // the sum accumulates atomically
    launch_sumsq(R, n, p, ldr, dsum, nsm, st);
    double obj = 0.0;
    if (cudaMemcpyAsync(&obj, dsum, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      MSE_FAIL(GODEC_ERR_CUDA, "objective read-back failed");
    if (history) history[t] = obj;
  }
  if (C) {
    cudaMemsetAsync(C, 0, (size_t)k * r_stride * p * sizeof(float), st);
    for (int j = 0; j < k; ++j) launch_transpose(V[j], p, r_eff[j], r_eff[j], C + (size_t)j * r_stride * p, p, st);
  }
  if (Lsum) {
    launch_sub(X, ldx, R, ldr, n, p, Lsum, ldl, nsm, st);
    launch_sparse_axpy(Lsum, ldl, p, Si[0], Sv[0], nnz_cur, -1.f, nsm, st);
  }
  if (nnz) *nnz = nnz_cur;
  if (S_idx && S_val && S_cap >= nnz_cur && nnz_cur > 0) {
    cudaMemcpyAsync(S_idx, Si[0], (size_t)nnz_cur * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(S_val, Sv[0], (size_t)nnz_cur * 4, cudaMemcpyDeviceToDevice, st);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) MSE_FAIL(GODEC_ERR_CUDA, "%s", cudaGetErrorString(e));
  const bool short_cap = (S_idx || S_val) && S_cap < nnz_cur;
  cleanup();
#undef MSE_FAIL
  if (short_cap) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mse_train: S_cap %lld < nnz %lld", (long long)S_cap,
             (long long)nnz_cur);
    return GODEC_ERR_ARG;
  }
  return GODEC_OK;
}

godec_status godec_grebsmo_run(godec_ctx* c, int32_t* r_out, double* stage_err, int32_t cap, int32_t* n_stages) {
  if (!c || !c->greb) {
    if (c) fail(c, GODEC_ERR_STATE, "godec_grebsmo_run needs a context from godec_grebsmo_init");
    return c ? GODEC_ERR_STATE : GODEC_ERR_ARG;
  }
  godec_status s = reset_state(c);
  if (s) return s;
  const int64_t m = c->p.m, n = c->p.n;
  const int RP = c->RP;
  const size_t rr = (size_t)RP * RP;
  cudaStream_t st = c->st;
  launch_fill_zero(c->V, (size_t)n * RP * sizeof(float), st);
  launch_fill_zero(c->Q2, (size_t)n * RP * sizeof(float), st);
  launch_fill_zero(c->Q1, (size_t)m * RP * sizeof(float), st);
  launch_fill_zero(c->U, (size_t)m * RP * sizeof(float), st);
  launch_fill_zero(c->P, (size_t)std::max(m, n) * RP * sizeof(float), st);
  launch_fill_zero(c->Qa, (size_t)m * 64 * sizeof(float), st);
  launch_fill_zero(c->Qb, (size_t)n * 64 * sizeof(float), st);
  // Reading of eq. softt on the GPU: S is nonzero where |R| > lambda, i.e. where the key
  // (bits of |R|) exceeds that of (float) lambda.
  const float lamf = (float)c->gp.lambda;
  unsigned guess;
  memcpy(&guess, &lamf, sizeof(guess));
  guess += 1u;
  int ri = std::min(c->gp.dr, c->gp.r_max), stage = 0, nst = 0;
  c->r = ri;
  greb_increment(c, 0, ri, 0);   // Reading R18: the first V from X itself
  CK(cudaGetLastError());
  for (;;) {
    c->r = ri;
    for (int k = 0; k < c->gp.K; ++k) {
      greb_lstep(c, ri);
      for (int attempt = 0;; ++attempt) {
        greb_sstep(c, ri, guess, c->Q1, (float)c->gp.lambda);
        CK(cudaGetLastError());
        Ctl h;
        if ((s = read_ctl(c, &h))) return s;
        if (h.timeout) return fail(c, GODEC_ERR_TIMEOUT, "a device-side wait of the tensor-core product timed out");
        if (h.nonfinite) return fail(c, GODEC_ERR_NONFINITE, "non-finite values in X - U V");
        if (h.abort && h.need_bigger_cand && attempt < 8) {
          if ((s = clear_counters(c))) return s;
          if ((s = rebuild_sbits(c))) return s;
          if ((s = greb_grow(c, h, h.cand_count))) return s;
          continue;
        }
        if (h.abort) return fail(c, GODEC_ERR_STATE, "GreBsmo inner step aborted");
        if (h.range_err) {
          if ((s = rescale_z(c))) return s;
          if ((s = SET_CTL(range_err, 0))) return s;
        }
        break;
      }
    }
    Ctl h;
    if ((s = read_ctl(c, &h))) return s;
    if (stage_err && nst < cap) stage_err[nst] = h.rel_err;
    ++nst;
    if (h.rel_err <= c->gp.tau || ri >= c->gp.r_max) break;   // Reading R17
    const int add = std::min(c->gp.dr, c->gp.r_max - ri);
    ++stage;
    c->r = ri;
    greb_increment(c, ri, add, stage);
    ri += add;
  }
  // the factored form of L = U W^T = U diag(sigma) Vh^T: Vh = Qv Rv, M = diag(sigma) Rv^T
  // = Ur S Vr^T, L = (U Ur) S (Qv Vr)^T
  {
    const size_t q = (size_t)64 * 64;
    float *R1 = c->Rf, *T1 = R1 + q, *R2m = T1 + q, *T2 = R2m + q;
    c->r = ri;
    cqr2(c, c->V, n, ri, RP, c->Qb, R1, T1, R2m, T2);
    launch_rmul(R2m, R1, RP, ri, c->rf_core, 1, c->sigma, st);
    launch_fill_zero(c->U, (size_t)m * RP * sizeof(float), st);
    launch_fill_zero(c->V, (size_t)n * RP * sizeof(float), st);
    launch_fill_zero(c->sigma, (size_t)RP * sizeof(float), st);
    launch_svd_small(c->rf_core, ri, ri, c->rf_U, c->sigma, c->rf_V, st, nullptr, true);
    launch_tall_small_d(c->Q1, RP, ri, c->rf_U, ri, 0, ri, m, 1.f, 0.f, c->U, RP, st);
    launch_tall_small_d(c->Qb, RP, ri, c->rf_V, ri, 0, ri, n, 1.f, 0.f, c->V, RP, st);
    (void)rr;
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  if (r_out) *r_out = ri;
  if (n_stages) *n_stages = nst;
  return GODEC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Batched form: many independent problems of uneven m, n and r.  One batch iteration is
// one launch of one CUDA graph holding an iteration of every problem as a parallel
// branch, all on the exact-normaliser path: with lagged normalisers, problems shaped
// like the batched workload (2-5 % of entries in S, whose support moves between
// iterations) raised the normaliser alarm in nearly every iteration, and every change of
// path means capturing the whole batch graph again.  So the graph is captured once (and
// again only after a rank drop).  Each problem's grids are sized for a share of the SMs
// (its budget), so the branches' kernels run side by side and one problem's
// latency-bound r x r work overlaps another's streaming.  An autotuner picks the budget
// policy by timing the batch graph of each candidate on the problems themselves.
// ---------------------------------------------------------------------------------
struct godec_batch {
  std::vector<godec_ctx*> ctx;
  std::vector<int> sm;           // budget of each problem
  std::vector<int> graph_r;      // each problem's r when the graph was captured
  std::vector<unsigned> graph_epoch;   // each problem's graph epoch at the capture
  int recaptures = 0;            // batch graphs captured since init
  Ctl* hctl = nullptr;           // pinned host copies of the control blocks (count)
  cudaStream_t st = nullptr;     // the caller's stream
  cudaStream_t cap_st = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec = nullptr;
  int policy = 0;
  double policy_ms[GODEC_BATCH_POLICIES] = {};
  char err[200] = {0};
};

namespace {

godec_status bfail(godec_batch* b, godec_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->err, sizeof(b->err), fmt, ap);
  va_end(ap);
  return s;
}

// Size every grid of problem c for B SMs (the stream-K geometry of both product
// orientations and the S-step's grids).  The stream-K buffers were sized for the whole
// device at init; a smaller grid never needs more (fewer CTAs split each tile less).
godec_status set_budget(godec_ctx* c, int B) {
  B = std::max(1, std::min(B, c->nsm_dev));
  const TcGeom g0 = tc_geometry(c->p.m, c->p.n, B), g1 = tc_geometry(c->p.n, c->p.m, B);
  size_t npart = 0, npend = 0;
  for (const TcGeom& g : {g0, g1}) {
    npart = std::max(npart, (size_t)g.tiles * g.maxseg * 128 * c->RP);
    npend = std::max(npend, (size_t)g.G * g.maxpend);
  }
  if (npart > c->npart_cap || npend > c->npend_cap)
    return fail(c, GODEC_ERR_STATE, "budget %d needs larger stream-K buffers", B);
  c->nsm = B;
  c->tg[0] = g0;
  c->tg[1] = g1;
  free_graphs(c);
  return GODEC_OK;
}

// Budgets of policy k on N SMs: 0 gives every problem the whole device; 1..4 give problem i
// a share of the SMs proportional to its m n, oversubscribed 1, 2, 4 and 8 times (at least
// 4 SMs, at most all).
void budgets_of(int count, const int64_t* m, const int64_t* n, int N, int k, int* out) {
  double W = 0.0;
  for (int i = 0; i < count; ++i) W += (double)m[i] * (double)n[i];
  for (int i = 0; i < count; ++i) {
    if (k == 0) {
      out[i] = N;
      continue;
    }
    const double alpha = (double)(1 << (k - 1));
    const int B = (int)std::ceil(alpha * N * ((double)m[i] * (double)n[i]) / W);
    out[i] = std::max(std::min(4, N), std::min(N, B));
  }
}

void policy_budgets(const godec_batch* b, int k, std::vector<int>& out) {
  std::vector<int64_t> m(b->ctx.size()), n(b->ctx.size());
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    m[i] = b->ctx[i]->p.m;
    n[i] = b->ctx[i]->p.n;
  }
  out.resize(b->ctx.size());
  budgets_of((int)b->ctx.size(), m.data(), n.data(), b->ctx[0]->nsm_dev, k, out.data());
}

godec_status apply_budgets(godec_batch* b, const std::vector<int>& bud) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    godec_status s = set_budget(b->ctx[i], bud[i]);
    if (s) return bfail(b, s, "problem %zu: %s", i, b->ctx[i]->err);
  }
  b->sm = bud;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  return GODEC_OK;
}

// Capture one iteration of every problem, each a branch forked from and joined into the
// batch's capture stream.
godec_status build_batch_graph(godec_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return bfail(b, GODEC_ERR_CUDA, "stream synchronize failed");
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->cap_st);
  for (size_t i = 0; i < b->ctx.size() && e == cudaSuccess; ++i) {
    godec_ctx* c = b->ctx[i];
    cudaStream_t user = c->st;
    c->st = c->cap_st;
    e = cudaStreamWaitEvent(c->st, b->fork, 0);
    if (e == cudaSuccess) {
      enqueue_iteration(c, false);
      e = cudaEventRecord(b->join[i], c->st);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_st, b->join[i], 0);
    c->st = user;
  }
  cudaError_t e2 = cudaStreamEndCapture(b->cap_st, &g);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, GODEC_ERR_CUDA, "batch graph capture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, GODEC_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  b->graph_r.resize(b->ctx.size());
  b->graph_epoch.resize(b->ctx.size());
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    b->graph_r[i] = b->ctx[i]->r;
    b->graph_epoch[i] = b->ctx[i]->graph_epoch;
  }
  ++b->recaptures;
  return GODEC_OK;
}

// Control blocks of every problem: one copy each into pinned memory, one synchronise.
godec_status read_all(godec_batch* b) {
  for (size_t i = 0; i < b->ctx.size(); ++i)
    if (cudaMemcpyAsync(&b->hctl[i], b->ctx[i]->ctl, offsetof(Ctl, hist), cudaMemcpyDeviceToHost, b->st) !=
        cudaSuccess)
      return bfail(b, GODEC_ERR_CUDA, "control block copy failed");
  if (cudaStreamSynchronize(b->st) != cudaSuccess)
    return bfail(b, GODEC_ERR_CUDA, "batch iteration: %s", cudaGetErrorString(cudaGetLastError()));
  return GODEC_OK;
}

godec_status batch_reset(godec_batch* b) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    godec_status s = reset_state(b->ctx[i]);
    if (s) return bfail(b, s, "problem %zu: %s", i, b->ctx[i]->err);
  }
  return GODEC_OK;
}

// n_iter launches of the batch graph; then a problem whose iteration aborted in the graph
// (its later launches skipped it) is handled and catches up on its own graphs.
godec_status batch_iterate(godec_batch* b, int n_iter) {
  if (n_iter <= 0) return GODEC_OK;
  const size_t P = b->ctx.size();
  godec_status s = read_all(b);
  if (s) return s;
  std::vector<char> out(P);   // sits out: converged or failed before this call
  std::vector<int> before(P);
  bool rebuild = !b->gexec;
  for (size_t i = 0; i < P; ++i) {
    out[i] = b->hctl[i].abort ? 1 : 0;
    before[i] = b->hctl[i].iter;
    // a rank drop, a candidate buffer grown, a new budget or a reset: the captured
    // graph holds stale sizes or pointers of that problem
    rebuild = rebuild || b->graph_r[i] != b->ctx[i]->r || b->graph_epoch[i] != b->ctx[i]->graph_epoch;
  }
  if (rebuild && (s = build_batch_graph(b))) return s;
  for (int t = 0; t < n_iter; ++t)
    if (cudaGraphLaunch(b->gexec, b->st) != cudaSuccess) return bfail(b, GODEC_ERR_CUDA, "batch graph launch failed");
  if ((s = read_all(b))) return s;
  for (size_t i = 0; i < P; ++i) {
    if (out[i]) continue;
    godec_ctx* c = b->ctx[i];
    const Ctl& h = b->hctl[i];
    const int done = h.iter - before[i];
    c->exact_iters += done;
    if (done < n_iter) {
      if (!h.abort) return bfail(b, GODEC_ERR_STATE, "problem %zu: %d of %d iterations ran", i, done, n_iter);
      if (h.converged) continue;
      if ((s = handle_abort(c, h)) || (s = run_iterations(c, n_iter - done, -1.0)))
        return bfail(b, s, "problem %zu: %s", i, c->err);
    }
  }
  return GODEC_OK;
}

void batch_free(godec_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (godec_ctx* c : b->ctx) godec_destroy(c);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  if (b->hctl) cudaFreeHost(b->hctl);
  delete b;
}

}  // namespace

extern "C" {

godec_status godec_batch_init(godec_batch** out, int32_t count, const godec_params* params, const float* const* X,
                              const float* const* A1, int32_t flags, void* stream) {
  if (!out) return GODEC_ERR_ARG;
  *out = nullptr;
  if (count < 1 || count > GODEC_BATCH_MAX || !params || !X || !A1) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_batch_init: need 1 <= count <= %d and non-NULL arrays",
             GODEC_BATCH_MAX);
    return GODEC_ERR_ARG;
  }
  for (int i = 0; i < count; ++i)
    if (params[i].precision != GODEC_PREC_FP32) {
      snprintf(g_static_err, sizeof(g_static_err), "godec_batch_init: problem %d: the batched form is float32", i);
      return GODEC_ERR_ARG;
    }
  godec_batch* b = new (std::nothrow) godec_batch;
  if (!b) return GODEC_ERR_OOM;
  b->st = reinterpret_cast<cudaStream_t>(stream);
  auto bail = [&](godec_status s, const char* why) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_batch_init: %.180s", why);
    batch_free(b);
    return s;
  };
  if (cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(GODEC_ERR_CUDA, "stream or event creation failed");
  if (cudaMallocHost(reinterpret_cast<void**>(&b->hctl), (size_t)count * sizeof(Ctl)) != cudaSuccess)
    return bail(GODEC_ERR_OOM, "pinned control blocks");
  b->join.assign(count, nullptr);
  b->ctx.reserve(count);
  for (int i = 0; i < count; ++i) {
    if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
      return bail(GODEC_ERR_CUDA, "event creation failed");
    godec_ctx* c = nullptr;
    godec_status s = godec_init(&c, &params[i], X[i], A1[i], stream);
    if (s) {
      char why[200];
      snprintf(why, sizeof(why), "problem %d: %.150s", i, g_static_err);
      return bail(s, why);
    }
    b->ctx.push_back(c);
  }
  std::vector<int> bud;
  if (flags & GODEC_BATCH_NO_TUNE) {
    policy_budgets(b, 0, bud);
    if (apply_budgets(b, bud)) return bail(GODEC_ERR_STATE, b->err);
    b->policy = 0;
  } else {
    // time 3 batch iterations of each policy after two warm-up ones (the first takes the
    // exact path, the second the path the problems then keep), from the initial state
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return bail(GODEC_ERR_CUDA, "event creation failed");
    double best = 0.0;
    int best_k = 0;
    godec_status s = GODEC_OK;
    for (int k = 0; k < GODEC_BATCH_POLICIES && !s; ++k) {
      policy_budgets(b, k, bud);
      if ((s = apply_budgets(b, bud)) || (s = batch_iterate(b, 2))) break;
      cudaEventRecord(e0, b->st);
      for (int t = 0; t < 3; ++t) cudaGraphLaunch(b->gexec, b->st);
      cudaEventRecord(e1, b->st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        s = bfail(b, GODEC_ERR_CUDA, "tuning launch failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      b->policy_ms[k] = ms / 3.0;
      if (k == 0 || b->policy_ms[k] < best) {
        best = b->policy_ms[k];
        best_k = k;
      }
      s = batch_reset(b);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return bail(s, b->err);
    policy_budgets(b, best_k, bud);
    if (apply_budgets(b, bud) || batch_reset(b)) return bail(GODEC_ERR_STATE, b->err);
    b->policy = best_k;
  }
  *out = b;
  return GODEC_OK;
}

godec_status godec_batch_iterate(godec_batch* b, int32_t n_iter) {
  if (!b) return GODEC_ERR_ARG;
  if (n_iter < 0) return bfail(b, GODEC_ERR_ARG, "n_iter must be >= 0");
  return batch_iterate(b, n_iter);
}

godec_status godec_batch_reset(godec_batch* b) {
  if (!b) return GODEC_ERR_ARG;
  return batch_reset(b);
}

godec_ctx* godec_batch_problem(godec_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

godec_status godec_batch_tuning(godec_batch* b, int32_t* sm, double* policy_ms, int32_t* policy,
                                int32_t* recaptures) {
  if (!b) return GODEC_ERR_ARG;
  if (recaptures) *recaptures = b->recaptures;
  if (sm)
    for (size_t i = 0; i < b->sm.size(); ++i) sm[i] = b->sm[i];
  if (policy_ms)
    for (int k = 0; k < GODEC_BATCH_POLICIES; ++k) policy_ms[k] = b->policy_ms[k];
  if (policy) *policy = b->policy;
  return GODEC_OK;
}

void godec_batch_destroy(godec_batch* b) { batch_free(b); }

godec_status godec_batch_budgets(int32_t count, const int64_t* m, const int64_t* n, int32_t nsm, int32_t policy,
                                 int32_t* sm) {
  if (count < 1 || !m || !n || !sm || nsm < 1 || policy < 0 || policy >= GODEC_BATCH_POLICIES)
    return GODEC_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (m[i] < 1 || n[i] < 1) return GODEC_ERR_ARG;
  std::vector<int> out(count);
  budgets_of(count, m, n, nsm, policy, out.data());
  for (int i = 0; i < count; ++i) sm[i] = out[i];
  return GODEC_OK;
}

godec_status godec_tc_geometry(int64_t rows, int64_t K, int32_t nsm, int64_t* out) {
  if (rows < 1 || K < 1 || nsm < 1 || !out) return GODEC_ERR_ARG;
  const TcGeom g = tc_geometry(rows, K, nsm);
  out[0] = g.tiles;
  out[1] = g.ks;
  out[2] = g.S;
  out[3] = g.G;
  out[4] = g.maxseg;
  out[5] = g.maxpend;
  return GODEC_OK;
}

const char* godec_batch_last_error(godec_batch* b) { return b ? b->err : g_static_err; }

}  // extern "C"
