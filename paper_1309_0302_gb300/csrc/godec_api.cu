// Host side of the C ABI declared in include/godec.h: context and workspace,
// the launch sequence of one iteration of Algorithm 1 (captured once into a
// CUDA graph and replayed), recovery from aborted iterations (rank drop,
// candidate overflow), and the result getters.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "godec_internal.cuh"

using namespace godec;

struct godec_ctx {
  godec_params p;
  int r = 0;          // current rank (drops after a failed rank test)
  int RP = 0;         // padded width of the skinny buffers (from the initial r)
  cudaStream_t st = nullptr;
  cudaStream_t cap_st = nullptr;   // private stream used only while capturing the graph
  int dev = 0, nsm = 0;
  const float* X = nullptr;
  float* Z = nullptr;
  int64_t ldz = 0;
  void* Z16 = nullptr;
  float* A1 = nullptr;                 // n x RP; columns >= r kept at zero
  float* A1_orig = nullptr;            // n x RP as given (restored by godec_reset)
  float* P = nullptr;                  // max(m,n) x RP
  float* Qb[2] = {nullptr, nullptr};   // max(m,n) x RP
  float* Q1 = nullptr;                 // m x RP
  float* Q2 = nullptr;                 // n x RP
  float* U = nullptr;                  // m x RP
  float* V = nullptr;                  // n x RP
  float* sigma = nullptr;              // RP
  float* Um = nullptr;
  float* Vm = nullptr;
  float* Rm = nullptr;
  float* Rinv = nullptr;
  float* M = nullptr;
  float* part = nullptr;
  size_t part_elems = 0;
  void* gram = nullptr;
  Ctl* ctl = nullptr;
  unsigned* cand_key = nullptr;
  long long* cand_idx = nullptr;
  float* cand_val = nullptr;
  unsigned long long cap = 0;
  long long* S_idx[2] = {nullptr, nullptr};
  float* S_val[2] = {nullptr, nullptr};
  int idx_bits = 1;
  cudaGraphExec_t gexec = nullptr;
  int graph_r = -1;
  double tol_in_graph = -2.0;
  int rank_drops = 0;
  int graph_nodes = 0;
  // kernel-level profiling (eager launches bracketed by events)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> prof_cls;      // class of event pair i
  size_t prof_used = 0;
  char err[200] = {0};
};

// Bracket one kernel launch with events when profiling (eager mode only).
#define PROF(c, cls, stmt)                                      \
  do {                                                          \
    if ((c)->prof) prof_mark(c, cls);                           \
    stmt;                                                       \
    if ((c)->prof) prof_mark(c, -1);                            \
  } while (0)

static void prof_mark(godec_ctx* c, int cls) {
  if (c->prof_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[c->prof_used++], c->st);
  if (cls >= 0) c->prof_cls.push_back(cls);
}

namespace {

const char* kStatusNames[] = {"ok", "invalid argument", "CUDA error", "out of memory",
                              "non-finite values", "device wait timed out", "invalid state",
                              "unsupported"};

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

void free_graph(godec_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->graph_r = -1;
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

// S-step of one iteration (Algorithm 1 line 9) on the current L factors; r = 0 means L = 0.
void enqueue_sstep(godec_ctx* c, int r) {
  const int64_t m = c->p.m, n = c->p.n;
  const int RP = c->RP;
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
  ra.RP = RP;
  ra.ctl = c->ctl;
  ra.cand_key = c->cand_key;
  ra.cand_idx = c->cand_idx;
  ra.cand_val = c->cand_val;
  ra.cand_cap = c->cap;
  for (int pass = 0; pass < 3; ++pass) {
    ra.pass = pass;
    PROF(c, 5, launch_residual(ra, c->nsm, st));
    PROF(c, 6, launch_after_pass(c->ctl, pass, c->p.k, c->cap, st));
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
    PROF(c, 7, launch_select_round(se, c->nsm, st));
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
  ea.Z16 = c->Z16;
  PROF(c, 8, launch_emit(ea, c->nsm, st));
  if (c->Z) PROF(c, 9, launch_z_update(ea, c->nsm, st));
}

// ---------------------------------------------------------------------------------
// One iteration of Algorithm 1 as a launch sequence on c->st.
// ---------------------------------------------------------------------------------
void enqueue_iteration(godec_ctx* c) {
  const int q = c->p.q, r = c->r, RP = c->RP;
  const int64_t m = c->p.m, n = c->p.n;
  cudaStream_t st = c->st;
  const int nprod = 6 * q + 3;
  const int i_q2 = 4 * q + 1;      // last product of L~^T Y1: Q2 = orth(Y2)
  const int i_rank = 4 * q + 2;    // first product of L~ Q2: rank test, start of M
  const float* B = c->A1;
  for (int i = 0; i < nprod; ++i) {
    const int trans = i & 1;
    const int64_t outdim = trans ? n : m, K = trans ? m : n;
    PassArgs pa{};
    pa.Z = c->Z;
    pa.bf16 = 0;
    pa.m = m;
    pa.n = n;
    pa.ldz = c->ldz;
    pa.B = B;
    pa.part = c->part;
    pass_geometry(outdim, K, c->nsm, &pa.splits, &pa.kchunk);
    pa.trans = trans;
    pa.RP = RP;
    pa.ctl = c->ctl;
    PROF(c, 0, launch_pass(pa, st));
    const int gmode = (i == i_rank) ? 2 : 1;
    PROF(c, 1, launch_reduce(c->part, pa.splits, outdim, RP, c->P, c->gram, gmode, c->ctl, st));
    CholArgs ca{};
    ca.gram_part = c->gram;
    ca.gram_double = (gmode == 2);
    ca.nblk = reduce_blocks(outdim);
    ca.r = r;
    ca.RP = RP;
    ca.R = c->Rm;
    ca.Rinv = c->Rinv;
    ca.M = c->M;
    ca.accumulate = (i < i_rank) ? 0 : (i == i_rank ? 2 : 1);
    ca.rank_test = (i == i_rank);
    ca.rank_tol = c->p.rank_tol > 0 ? c->p.rank_tol : 1e-4;
    ca.ctl = c->ctl;
    PROF(c, 2, launch_chol(ca, st));
    const bool final_q = (i == i_q2) || (i == nprod - 1);
    float* dst = final_q ? c->P : c->Qb[i & 1];
    PROF(c, 3, launch_apply(c->P, outdim, RP, c->Rinv, 1, dst,
                            final_q ? reinterpret_cast<float*>(c->gram) : nullptr, c->ctl, st));
    if (final_q) {
      // second CholeskyQR round for an orthonormal Q2 / Q1
      CholArgs cb = ca;
      cb.gram_double = 0;
      cb.rank_test = 0;
      cb.accumulate = (i == nprod - 1) ? 1 : 0;
      PROF(c, 2, launch_chol(cb, st));
      float* fin = (i == i_q2) ? c->Q2 : c->Q1;
      PROF(c, 3, launch_apply(c->P, outdim, RP, c->Rinv, 1, fin, nullptr, c->ctl, st));
      B = fin;
    } else {
      B = dst;
    }
  }
  // r x r core: SVD and singular-value root, then L = (Q1 Um) diag(sigma) (Q2 Vm)^T
  SvdArgs sa{};
  sa.M = c->M;
  sa.r = r;
  sa.RP = RP;
  sa.q = q;
  sa.Um = c->Um;
  sa.Vm = c->Vm;
  sa.sigma = c->sigma;
  sa.ctl = c->ctl;
  PROF(c, 4, launch_svd_root(sa, st));
  PROF(c, 3, launch_apply(c->Q1, m, RP, c->Um, 0, c->U, nullptr, c->ctl, st));
  PROF(c, 3, launch_apply(c->Q2, n, RP, c->Vm, 0, c->V, nullptr, c->ctl, st));

  enqueue_sstep(c, r);
}

godec_status build_graph(godec_ctx* c) {
  free_graph(c);
  cudaGraph_t g = nullptr;
  // The caller's stream may be the legacy default stream, which cannot be captured:
  // record on a private stream and launch the graph on the caller's stream.
  if (!c->cap_st) CK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
  CK(cudaStreamSynchronize(c->st));
  cudaStream_t user = c->st;
  c->st = c->cap_st;
  cudaError_t e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_iteration(c);
    e = cudaStreamEndCapture(c->st, &g);
  }
  c->st = user;
  if (e != cudaSuccess) return fail(c, GODEC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  c->graph_nodes = (int)nodes;
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(c, GODEC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graph_r = c->r;
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
  return GODEC_OK;
}

godec_status reset_state(godec_ctx* c) {
  free_graph(c);
  c->r = c->p.r;
  c->rank_drops = 0;
  if (c->A1_orig)
    CK(cudaMemcpyAsync(c->A1, c->A1_orig, (size_t)c->p.n * c->RP * sizeof(float), cudaMemcpyDeviceToDevice,
                       c->st));
  CK(cudaMemcpy2DAsync(c->Z, c->ldz * sizeof(float), c->X, c->p.ldx * sizeof(float),
                       c->p.n * sizeof(float), c->p.m, cudaMemcpyDeviceToDevice, c->st));
  Ctl h;
  memset(&h, 0, offsetof(Ctl, hist));
  h.k_req = c->p.k;
  h.k_eff = c->p.k;
  h.r_eff = c->p.r;
  h.tol = -1.0;
  CK(cudaMemcpyAsync(c->ctl, &h, offsetof(Ctl, hist), cudaMemcpyHostToDevice, c->st));
  launch_sumsq(c->X, c->p.m, c->p.n, c->p.ldx, reinterpret_cast<double*>(reinterpret_cast<char*>(c->ctl) +
               offsetof(Ctl, normX2)), c->nsm, c->st);
  launch_reset_iter(c->ctl, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return GODEC_OK;
}

// Run up to n graph launches, handling aborted iterations; stop early on convergence
// when tol >= 0.  *done receives the committed iterations.
godec_status run_iterations(godec_ctx* c, int n_iter, double tol, int* done) {
  *done = 0;
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  const int start = h.iter;
  if (h.tol != tol) {
    if ((s = SET_CTL(tol, tol))) return s;
  }
  int guard = 0;
  int chunk = tol >= 0.0 ? 1 : n_iter;
  while (*done < n_iter) {
    if (!c->gexec || c->graph_r != c->r) {
      if ((s = build_graph(c))) return s;
    }
    const int want = std::min(chunk, n_iter - *done);
    for (int i = 0; i < want; ++i) CK(cudaGraphLaunch(c->gexec, c->st));
    if ((s = read_ctl(c, &h))) return s;
    *done = h.iter - start;
    if (h.abort) {
      if (h.converged) return GODEC_OK;
      if (h.nonfinite) {
        launch_reset_iter(c->ctl, c->st);
        return fail(c, GODEC_ERR_NONFINITE, "non-finite values in X - L (iteration %d)", h.iter + 1);
      }
      if (h.rank_drop) {
        c->r = h.r_eff;
        ++c->rank_drops;
        if (c->r <= 0) return fail(c, GODEC_ERR_UNSUPPORTED, "rank test found rank 0 (X - S is zero)");
        if ((s = drop_columns(c))) return s;
      } else if (h.need_bigger_cand) {
        unsigned long long cap = c->cap * 2;
        const unsigned long long mn = (unsigned long long)(c->p.m * c->p.n);
        if (cap > mn) cap = mn;
        if (cap <= c->cap) return fail(c, GODEC_ERR_STATE, "candidate buffer cannot grow");
        free_graph(c);
        if ((s = alloc_candidates(c, cap))) return s;
      } else if (h.chol_fail) {
        return fail(c, GODEC_ERR_NONFINITE, "Cholesky breakdown in the power chain");
      }
      launch_reset_iter(c->ctl, c->st);
      CK(cudaGetLastError());
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
  if ((double)p->m * (double)p->n >= 281474976710656.0) { snprintf(why, nwhy, "m*n must be below 2^48"); return true; }
  return false;
}

char g_static_err[256];

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
  free_graph(c);
  void* ptrs[] = {c->Z, c->Z16, c->A1, c->A1_orig, c->P, c->Qb[0], c->Qb[1], c->Q1, c->Q2, c->U, c->V,
                  c->sigma, c->Um, c->Vm, c->Rm, c->Rinv, c->M, c->part, c->gram, c->ctl,
                  c->cand_key, c->cand_idx, c->cand_val, c->S_idx[0], c->S_idx[1],
                  c->S_val[0], c->S_val[1]};
  for (void* p : ptrs) cudaFree(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->cap_st) cudaStreamDestroy(c->cap_st);
  delete c;
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
  if (p->precision == GODEC_PREC_BF16_REFINE) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_init: the bf16 precision form is not built in this library");
    return GODEC_ERR_UNSUPPORTED;
  }
  godec_ctx* c = new (std::nothrow) godec_ctx;
  if (!c) return GODEC_ERR_OOM;
  c->p = *p;
  c->r = p->r;
  c->RP = round_up(p->r, 8);
  c->st = reinterpret_cast<cudaStream_t>(stream);
  auto bail = [&](godec_status s) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_init: %s", c->err);
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
  CKI(prepare_small_kernels());
  CKI(prepare_select_kernels());
  const int64_t m = p->m, n = p->n, mx = std::max(m, n);
  const int RP = c->RP;
  c->X = X;
  c->ldz = (n + 3) / 4 * 4;
  CKI(dalloc(&c->Z, (size_t)m * c->ldz));
  CKI(dalloc(&c->A1, (size_t)n * RP));
  CKI(dalloc(&c->P, (size_t)mx * RP));
  CKI(dalloc(&c->Qb[0], (size_t)mx * RP));
  CKI(dalloc(&c->Qb[1], (size_t)mx * RP));
  CKI(dalloc(&c->Q1, (size_t)m * RP));
  CKI(dalloc(&c->Q2, (size_t)n * RP));
  CKI(dalloc(&c->U, (size_t)m * RP));
  CKI(dalloc(&c->V, (size_t)n * RP));
  CKI(dalloc(&c->sigma, (size_t)RP));
  CKI(dalloc(&c->Um, (size_t)RP * RP));
  CKI(dalloc(&c->Vm, (size_t)RP * RP));
  CKI(dalloc(&c->Rm, (size_t)RP * RP));
  CKI(dalloc(&c->Rinv, (size_t)RP * RP));
  CKI(dalloc(&c->M, (size_t)RP * RP));
  int s1, s2;
  int64_t ch;
  pass_geometry(m, n, c->nsm, &s1, &ch);
  pass_geometry(n, m, c->nsm, &s2, &ch);
  c->part_elems = (size_t)std::max<int64_t>((int64_t)s1 * m, (int64_t)s2 * n) * RP;
  CKI(dalloc(&c->part, c->part_elems));
  // float64 Gram partials of every 64-row block, plus the reduced matrix
  CKI(dalloc(reinterpret_cast<double**>(&c->gram), (size_t)(reduce_blocks(mx) + 1) * RP * RP));
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
  c->idx_bits = 1;
  while ((1ull << c->idx_bits) < mn) ++c->idx_bits;
  launch_fill_zero(c->Q1, (size_t)m * RP * sizeof(float), c->st);
  launch_fill_zero(c->U, (size_t)m * RP * sizeof(float), c->st);
  CKI(dalloc(&c->A1_orig, (size_t)n * RP));
  launch_pad_copy(A1, n, p->r, p->r, c->A1_orig, RP, c->st);
  CKI(cudaGetLastError());
  godec_status s = reset_state(c);
  if (s) return bail(s);
  *out = c;
  return GODEC_OK;
#undef CKI
}

godec_status godec_reset(godec_ctx* c) {
  if (!c) return GODEC_ERR_ARG;
  return reset_state(c);
}

godec_status godec_iterate(godec_ctx* c, int32_t n_iter, double* rel_err) {
  if (!c) return GODEC_ERR_ARG;
  if (n_iter < 0) return fail(c, GODEC_ERR_ARG, "n_iter must be >= 0");
  int done = 0;
  godec_status s = run_iterations(c, n_iter, -1.0, &done);
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
  Ctl h;
  godec_status s = read_ctl(c, &h);
  if (s) return s;
  const int remaining = c->p.max_iter - h.iter;
  int done = 0;
  if (remaining > 0) {
    s = run_iterations(c, remaining, c->p.tol, &done);
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

godec_status godec_profile(godec_ctx* c, int32_t n_iter, double* ms, int64_t* launches,
                           double* bytes_product) {
  if (!c || n_iter < 0) return GODEC_ERR_ARG;
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
    c->prof = true;
    c->prof_used = 0;
    c->prof_cls.clear();
    enqueue_iteration(c);
    c->prof = false;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    for (size_t i = 0; i < c->prof_cls.size(); ++i) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
      const int k = c->prof_cls[i];
      if (ms) ms[k] += t;
      if (launches) launches[k] += 1;
    }
    if ((s = read_ctl(c, &h))) return s;
    if (h.abort) {
      if (h.nonfinite) return fail(c, GODEC_ERR_NONFINITE, "non-finite values");
      if (h.rank_drop) {
        c->r = h.r_eff;
        ++c->rank_drops;
        if (c->r <= 0) return fail(c, GODEC_ERR_UNSUPPORTED, "rank test found rank 0 (X - S is zero)");
        if ((s = drop_columns(c))) return s;
      } else if (h.need_bigger_cand) {
        unsigned long long cap = std::min<unsigned long long>(c->cap * 2, (unsigned long long)(c->p.m * c->p.n));
        free_graph(c);
        if ((s = alloc_candidates(c, cap))) return s;
      } else if (!h.converged) {
        return fail(c, GODEC_ERR_STATE, "aborted iteration while profiling");
      }
      launch_reset_iter(c->ctl, c->st);
      if (++guard > 64) return fail(c, GODEC_ERR_STATE, "too many aborted iterations");
      if ((s = read_ctl(c, &h))) return s;
    }
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
  info->reserved = 0;
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
  godec_ctx* c = nullptr;   // for CK's error path (no context yet)
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
  if (s && c) snprintf(g_static_err, sizeof(g_static_err), "godec_run_host: %s", c->err);
  godec_destroy(c);
  void* ptrs[] = {dX, dA, dU, dV, dS, dSi, dSv};
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, st);
  cudaStreamSynchronize(st);
  return s;
#undef CKH
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
  const int64_t outdim = trans ? n : m, K = trans ? m : n;
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int splits;
  int64_t kchunk;
  pass_geometry(outdim, K, nsm, &splits, &kchunk);
  float *Bp = nullptr, *part = nullptr, *Yp = nullptr;
  size_t bytes_b = (size_t)K * RP * sizeof(float), bytes_p = (size_t)splits * outdim * RP * sizeof(float),
         bytes_y = (size_t)outdim * RP * sizeof(float);
  if (cudaMallocAsync(reinterpret_cast<void**>(&Bp), bytes_b, st) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&part), bytes_p, st) != cudaSuccess ||
      cudaMallocAsync(reinterpret_cast<void**>(&Yp), bytes_y, st) != cudaSuccess) {
    if (Bp) cudaFreeAsync(Bp, st);
    if (part) cudaFreeAsync(part, st);
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: out of device memory");
    return GODEC_ERR_OOM;
  }
  launch_pad_copy(B, K, r, r, Bp, RP, st);
  PassArgs pa{};
  pa.Z = Z;
  pa.m = m;
  pa.n = n;
  pa.ldz = ldz;
  pa.B = Bp;
  pa.part = part;
  pa.splits = splits;
  pa.kchunk = kchunk;
  pa.trans = trans;
  pa.RP = RP;
  launch_pass(pa, st);
  launch_reduce(part, splits, outdim, RP, Yp, nullptr, 0, nullptr, st);
  launch_unpad_copy(Yp, outdim, RP, Y, r, st);
  cudaFreeAsync(Bp, st);
  cudaFreeAsync(part, st);
  cudaFreeAsync(Yp, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(g_static_err, sizeof(g_static_err), "godec_mul: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  return GODEC_OK;
}

godec_status godec_hard_threshold(const float* R, int64_t m, int64_t n, int64_t ldr, int64_t k,
                                  int64_t* idx, float* val, int64_t cap, int64_t* nnz, void* stream) {
  // A context with r = 0 (L = 0) and no working copy of X - S: only the S-step runs.
  if (!R || m < 1 || n < 1 || ldr < n || (ldr * 4) % 16 || k < 0 || k > m * n ||
      (reinterpret_cast<uintptr_t>(R) & 15)) {
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
  if (s) snprintf(g_static_err, sizeof(g_static_err), "godec_hard_threshold: %s", c->err);
  godec_destroy(c);
  return s;
}

godec_status godec_mul_ZB(const float* Z, int64_t m, int64_t n, int64_t ldz, const float* B, int32_t r,
                          float* Y, void* stream) {
  return mul_common(Z, m, n, ldz, B, r, Y, stream, 0);
}

godec_status godec_mul_ZtC(const float* Z, int64_t m, int64_t n, int64_t ldz, const float* C, int32_t r,
                           float* W, void* stream) {
  return mul_common(Z, m, n, ldz, C, r, W, stream, 1);
}

}  // extern "C"
