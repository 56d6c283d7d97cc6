// Internal declarations of the GoDec-BRP CUDA library (sm_103a).
//
// Data layout in HBM (row-major everywhere):
//   X   m x ldx  float32   borrowed input
//   Z   m x ldz  float32   working copy of X - S_{t-1}, updated sparsely
//   skinny m x RP / n x RP float32 factors, RP = r rounded up to 8 (<= 64);
//         padded columns are kept at zero
//   S   COO (int64 linear index, float32 value), double-buffered
//   candidates  (uint32 key, int64 index, float32 value) of the S-step
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/godec.h"

namespace godec {

// Block-uniform early exit of a kernel launched inside an iteration that may have been
// abandoned (flag = &ctl->abort; NULL never skips): thread 0 reads the flag once, since
// another stream may set it while the block runs.
__device__ __forceinline__ bool block_skip(const int* flag) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = flag ? *reinterpret_cast<const volatile int*>(flag) : 0;
  __syncthreads();
  return s_skip != 0;
}

constexpr int kMaxRP = 64;          // maximum padded rank
// Scale of the orthonormalised skinny operands in their float16 split form.  Entries
// of a unit column are at most 1, and a lagged normaliser can leave a column far from
// unit norm before the alarm catches it, so no scale-up: float16 then holds columns of
// norm up to ~6e4, and the split keeps 22 bits down to magnitudes of 2^-14 (below that
// the error is an absolute 2^-35, negligible against a unit column).
constexpr float kSkinnyScale = 1.f;
// The working copy Z = (X - S) s_Z is kept below this magnitude (float16 holds 65504):
// s_Z puts max |X| in [2^12, 2^13), and an S-step that writes a larger entry flags
// range_err so Z is rescaled before the next product.
constexpr float kZRange = 32768.f;
constexpr int kHistBins = 4096;     // first radix digit: key bits 30..19
constexpr int kD1Shift = 19;
constexpr int kNumSelRounds = 7;    // 3 key digits + 4 index digits

// Pass modes of the residual (S-step) kernel.
enum PassMode : int { PASS_NONE = 0, PASS_FULL = 1, PASS_CAND = 2, PASS_DUMP = 3 };

// Device-resident control block shared by the kernels of one context.  Scalars come
// first so the host can read them with one small copy; histograms follow.
struct Ctl {
  // --- residual passes of the current S-step -------------------------------
  int plan[3];                  // mode of residual pass 0/1/2 this iteration
  unsigned guess[3];            // candidate threshold key per pass
  int passes_run;
  int ready;                    // candidates cover the top-k_eff keys
  int need_bigger_cand;         // candidate buffer too small for an exact bin
  int pad0;
  unsigned long long cand_count;
  long long k_req;              // k requested
  long long k_eff;              // min(k, #nonzero residuals) once known
  double sumsq_noncand;         // sum R^2 over entries that are not candidates
  double sumsq_full;            // sum R^2 over all entries (full-histogram pass)
  unsigned done_ctas;           // last-block counters
  unsigned done_ctas2;
  // --- exact selection over the candidates ----------------------------------
  unsigned long long key_prefix;
  unsigned long long idx_prefix;
  long long need;               // rank still to select inside the prefix
  unsigned tau_key;             // k-th largest key
  int key_done, idx_done;
  int pad1;
  unsigned long long idx_cut;   // ties selected up to this index (inclusive)
  // --- emit / objective -----------------------------------------------------
  unsigned long long nnz_new;
  double sumsq_cand_out;        // sum R^2 over candidates left out of Omega
  double obj, rel_err, normX2;
  double tol;                   // stop test threshold (< 0: disabled)
  unsigned next_guess;
  int cur;                      // which S buffer is current
  long long nnz_cur;            // |Omega| of the committed S
  long long nnz_prev;
  int iter;                     // committed iterations
  // --- L-step ----------------------------------------------------------------
  int r_eff;                    // rank found by the rank test (<= r)
  int rank_drop;                // the rank test lowered r (iteration aborted)
  int abort;                    // remaining kernels of the iteration are skipped
  int nonfinite;
  int chol_fail;
  int svd_sweeps;
  int converged;                // stop test met (sets abort, not an error)
  int last_passes;              // residual passes used by the last committed S-step
  int chol_shifts;              // Cholesky factorisations that needed a diagonal shift
  int alarm;                    // a lagged normaliser left the chain ill-conditioned
  int slot_parity;              // which half of the slot buffers holds this iteration's T
  int timeout;                  // a bounded device-side wait gave up
  double m_logscale;            // Pi (core of the last chain) is stored divided by exp(.)
  float zscale[2];              // power-of-two scale s_Z of the stored Z = (X - S) s_Z, and 1 / s_Z
  unsigned zmax_bits;           // scratch: max |Z| as float bits
  int range_err;                // the S-step wrote an entry of Z above kZRange (rescale Z before reuse)
  // --- histograms ------------------------------------------------------------
  unsigned hist[kHistBins];     // digit-1 histogram of |R| keys (full pass)
  unsigned sel_hist[kHistBins];
};

// --------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All take the context stream.
// --------------------------------------------------------------------------------

// Streaming product Y = Zsrc B (Zsrc rows x K row-major with stride ld, B K x RP)
// with split-K partials; the last CTA of each 128-row tile sums the partials (split
// order), right-multiplies by Tn (RP x RP, nullable), writes `out` (rows x RP) and the
// tile's Gram partial (gram_mode 0 none, 1 float, 2 exact products in double-float).
struct ProdArgs {
  const void* Z;
  int bf16;
  int64_t rows, K, ld;
  const float* B;
  float* part;             // splits x rows x RP
  int splits;
  int64_t kchunk;          // multiple of 32
  unsigned* counters;      // prod_tiles(rows) zeros; left at zero after the call
  float* out;
  const float* Tn[2];      // normaliser by slot parity (both null: none)
  void* gram_part;         // prod_tiles(rows) x RP x RP (float or double)
  int gram_mode;
  int RP;
  const Ctl* ctl;          // nullable; abort flag checked
};
void launch_prod(const ProdArgs& a, cudaStream_t st);
void prod_geometry(int64_t rows, int64_t K, int nsm, int* splits, int64_t* kchunk);
int64_t prod_tiles(int64_t rows);
cudaError_t prepare_stream_kernels();

// Q = P T with T dense RP x RP (T0 or T1 by the slot parity in ctl; T0 without ctl),
// optional float Gram partials of Q per apply_blocks() row block.  P and Q may alias;
// Q may be null.  With bt2 set, also writes the float16 split transposed operand of the
// tensor-core product, [c1^T; c2^T] (2 RP x ldb halves) with Q kSkinnyScale =
// c1 + 2^-11 c2.
void launch_apply(const float* P, int64_t rows, int RP, const float* T0, const float* T1, float* Q,
                  float* gram_part, const Ctl* ctl, cudaStream_t st, void* bt2 = nullptr, int64_t ldb = 0);

// First projection of the chain from the cached X A1 (k_sproj.cu): P = X A1 - S A1 (m x RP,
// row stride RP; XA1 and A1 likewise), S read on its support (bitmap ctl->cur of sbits,
// `words` words per bitmap) as X - Z / s_Z; each row's entries are subtracted in column
// order.  Like the product, it abandons the iteration when Z is flagged out of range.
void launch_sproj(const float* XA1, const float* A1, int RP, const float* X, int64_t ldx, const float* Z, int64_t ldz,
                  int64_t m, int64_t n, const unsigned* sbits, long long words, Ctl* ctl, float* P,
                  cudaStream_t st);

// Tensor-core streaming product (k_tc.cu).
struct TcGeom {
  int64_t tiles = 0, ks = 0, S = 0;
  int G = 0, maxseg = 0;
  int maxpend = 0;           // completions one CTA may owe (list entries per CTA)
};
TcGeom tc_geometry(int64_t rows, int64_t K, int nsm);
int tc_rpp(int RP);
// Float16 split transposed operand of a row-major rows x RP matrix B (2 RP x ldb
// halves), each column scaled by a power of two; cscale (RP) receives the factors that
// undo the scaling.
void launch_split_t(const float* B, int64_t rows, int RP, void* bt2, int64_t ldb, float* cscale, cudaStream_t st,
                    const int* skip = nullptr);
// zscale = {s, 1/s}: the power of two with max |Z| s in [2^12, 2^13) (1 if Z is zero or
// not finite); zmax is scratch.
void launch_zscale(const float* Z, int64_t rows, int64_t cols, int64_t ld, unsigned* zmax, float* zscale, int nsm,
                   cudaStream_t st);
// dst = src * scale[0] (rows x cols, strides lds / ldd); dst may equal src.
void launch_scale_copy(const float* src, int64_t rows, int64_t cols, int64_t lds, float* dst, int64_t ldd,
                       const float* scale, int nsm, cudaStream_t st);
// zscale[0..1] *= f[0..1] (one thread).
void launch_scale_update(float* zscale, const float* f, cudaStream_t st);
bool make_tmap_f32(void* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows);
bool make_tmap_f16(void* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows);
cudaError_t prepare_tc_kernels();
struct TcLaunch {
  const void* mapA;        // CUtensorMap over Zsrc (rows x K), box 32 x 128
  const void* mapB;        // CUtensorMap over the float16 split operand (2 RP x K), box 64 x 2 RP
  int64_t rows, K;
  int RP;
  TcGeom geom;
  float* part;             // tiles x maxseg x 128 x RP
  unsigned* counters;      // tiles, zero
  float* out;              // rows x RP (nullable)
  void* bt2;               // 2 RP x ldb halves (nullable)
  int64_t ldb;
  const float* Tn[2];
  const float* cscale;     // per-column output factor (nullable)
  const float* zscale;     // {s_Z, 1/s_Z} on the device (nullable)
  int prescaled;           // Zsrc already holds x s_Z
  void* gram_part;
  int gram_mode;
  int t_upper;             // Tn upper triangular (inverse of an upper-triangular factor)
  int half_a;              // mapA is the float16 copy Z16 (box 64 halves x 128 rows)
  int* pend;               // G x geom.maxpend ints of scratch
  Ctl* ctl;
  int pdl = 0;             // programmatic dependent launch on the preceding kernel of the stream
  int z_prefetch = 0;      // the preceding kernels leave Zsrc unchanged: its first stages may be
                           // loaded before the wait on them (with pdl)
};
void launch_prod_tc(const TcLaunch& l, cudaStream_t st);
int64_t apply_blocks(int64_t rows);

// r x r kernels (k_small.cu).
// Gram partials of the 128-row tiles of the rows x RP float32 matrix Y (row stride RP;
// k_gram.cu): mode 1 float, mode 2 exactly accumulated double; layout as the product's
// gram_part.
void launch_gram_tiles(const float* Y, int64_t rows, int RP, int mode, void* part, const Ctl* ctl, cudaStream_t st);
void launch_gram_sum(const void* part, int gram_double, int64_t nblk, int RP, double* out, const Ctl* ctl,
                     cudaStream_t st, float* out32 = nullptr);
// R (upper, Rᵀ R = Gram) and T = R^{-1}, both RP x RP.
void launch_chol(const double* g64, int r, int RP, float* R, float* T, Ctl* ctl, cudaStream_t st,
                 float alarm_ratio = 0.f, bool fp64 = false, const float* g32 = nullptr);
struct SlotLaunch {
  const double* g64 = nullptr;
  const float* g32 = nullptr;   // float copy of g64 (nullable)
  int g_is_p = 0;
  const float* R_app[2] = {nullptr, nullptr};
  const float* T_app[2] = {nullptr, nullptr};
  const float* L1 = nullptr;
  const float* L2 = nullptr;
  float* R_next[2] = {nullptr, nullptr};
  float* T_next[2] = {nullptr, nullptr};
  float* Pi = nullptr;
  int pi_mode = 0;
  int fast = 0;
  int r = 0, RP = 0;
  float alarm_ratio = 30.f;
  Ctl* ctl = nullptr;
};
void launch_slot(const SlotLaunch& l, cudaStream_t st);
void launch_rank(const double* g64, int r, int RP, double rank_tol, Ctl* ctl, cudaStream_t st);
// Um is returned as Tl Um when Tl (upper triangular RP x RP) is given.
void launch_svd(const float* Ra, const float* Rb, const float* Rapp0, const float* Rapp1, const float* Pi,
                float* Vprev, int r, int RP, int q, float* Um, float* Vm, float* sigma, Ctl* ctl, cudaStream_t st,
                const float* Tl = nullptr);

// --- S-step ---------------------------------------------------------------------
struct ResidualArgs {
  const float* X;
  int64_t m, n, ldx;
  const float* U;          // m x RP (orthonormal columns)
  const float* sigma;      // RP
  const float* V;          // n x RP
  int r, RP;
  int pass;                // 0, 1, 2
  Ctl* ctl;
  unsigned* cand_key;
  long long* cand_idx;
  float* cand_val;
  unsigned long long cand_cap;
};
void launch_residual(const ResidualArgs& a, int nsm, cudaStream_t st);

// Tensor-core residual pass (k_resid.cu).  A and B hold the float16 split of
// U diag(sqrt(sigma s_Z)) and V diag(sqrt(sigma s_Z)), rows of 128 halves (64 high,
// 64 low; K padded to 64), written by launch_lsplit after each L-step.
void launch_lsplit(const float* U, const float* V, const float* sigma, int64_t m, int64_t n, int RP, int r,
                   const float* zscale, void* A, void* B, cudaStream_t st, const int* skip = nullptr);
struct ResidTcLaunch {
  ResidualArgs ra;         // X, m, n, pass, ctl and the candidate buffers are used
  const void* mapX;        // CUtensorMap over X (m x n float32), box 32 x 128
  const void* mapA;        // over A (m x 128 halves), box 64 x 128
  const void* mapB;        // over B (n x 128 halves), box 64 x 64
  const float* zscale;     // {s_Z, 1/s_Z}
  float* dump;             // non-null: write R densely (row stride ldd) instead of selecting
  int64_t ldd;
  int nsm;
};
void launch_resid_tc(const ResidTcLaunch& l, cudaStream_t st);
cudaError_t prepare_resid_kernels();
void launch_after_pass(Ctl* ctl, int pass, long long k, unsigned long long cap, cudaStream_t st);

struct SelectArgs {
  Ctl* ctl;
  const unsigned* cand_key;
  const long long* cand_idx;
  const float* cand_val;
  unsigned long long cand_cap;
  long long k;
  int round;
  int idx_bits;            // bits needed for linear indices (<= 42)
};
void launch_select_round(const SelectArgs& a, int nsm, cudaStream_t st);

struct EmitArgs {
  Ctl* ctl;
  const unsigned* cand_key;
  const long long* cand_idx;
  const float* cand_val;
  unsigned long long cand_cap;
  long long* S_idx[2];
  float* S_val[2];
  const float* X;
  int64_t n, ldx;
  float* Z;
  int64_t ldz;
  float* Zt;               // transposed copy (n x ldzt), nullable
  int64_t ldzt;
  void* Z16;               // nullable bf16 copies (same strides)
  void* Zt16;
  const float* zscale;     // Z and Zt are stored scaled by zscale[0]
  long long max_nnz;       // bound on the support of S (k): the z-update grid
  unsigned* sbits;         // two bitmaps of m n bits (nullable), sbits_words words apart: bitmap
  long long sbits_words;   // `cur` holds the support of the committed S, the other one is clear.
                           // The emit marks Omega_t in the clear one, the restore of Omega_{t-1}
                           // skips the entries marked there and clears the old bitmap.
};
void launch_emit(const EmitArgs& a, int nsm, cudaStream_t st);
// The support bitmap of the committed S (bitmap ctl->cur) from its index list, after both
// bitmaps were cleared (an S-step cut short may leave bits behind).
void launch_sbits_rebuild(unsigned* sbits, long long words, long long* const S_idx[2], const Ctl* ctl,
                          long long max_nnz, cudaStream_t st);
void launch_z_update(const EmitArgs& a, int nsm, cudaStream_t st);
// Reset the per-iteration S-step state (after an aborted iteration or at start).
void launch_reset_iter(Ctl* ctl, cudaStream_t st);
// One bounded wait that nothing completes; flags ctl->timeout / abort when it gives up.
void launch_wait_check(Ctl* ctl, uint32_t polls, cudaStream_t st);

// Error text returned by godec_last_error(NULL) for calls without a context.
void set_static_error(const char* fmt, ...);

// Kernel attributes (dynamic shared memory limits); call before launching or capturing.
cudaError_t prepare_small_kernels();
cudaError_t prepare_select_kernels();

// Tall x small and sparse kernels (k_backward.cu), shared by the differentiated form and
// the precision form's correction.
// C (a x b, float64, row stride ldo) = A^T B for tall A (rows x a, lda) and B (rows x b,
// ldb), a, b <= 64, over fixed row partitions of about 128 rows, at most G of them (part
// holds G x a x b doubles); deterministic.
void launch_cross_gram(const float* A, int64_t lda, int a, const float* B, int64_t ldb, int b, int64_t rows,
                       double* part, int G, double* out, int ldo, cudaStream_t st, const int* skip = nullptr);
// C (rows x c, ldc) = beta C + alpha A (rows x a, lda) Bm (a x c, ldbm; Bm^T if trans), a, c <= 64
void launch_tall_small_f(const float* A, int64_t lda, int a, const float* Bm, int ldbm, int trans, int c, int64_t rows,
                         float alpha, float beta, float* C, int64_t ldc, cudaStream_t st, const int* skip = nullptr);
void launch_tall_small_d(const float* A, int64_t lda, int a, const double* Bm, int ldbm, int trans, int c,
                         int64_t rows, float alpha, float beta, float* C, int64_t ldc, cudaStream_t st,
                         const int* skip = nullptr);
// Precision form (k_refine.cu): the bases [P | Q] of the correction; float16 copy of a
// float32 matrix; the 2r x 2r core Ra K Rb^T of the tangent-space correction; SVD of an
// n x n float64 matrix (n <= 64), leading r triplets.
// W (rows x ld, float32) = [P | Q | 0] for P, Q rows x r with row stride ldp (2r <= ld).
void launch_concat2(const float* P, const float* Q, int64_t ldp, int r, int64_t rows, float* W, int ld,
                    cudaStream_t st, const int* skip = nullptr);
void launch_to_half(const float* src, int64_t rows, int64_t cols, int64_t lds, void* dst, int64_t ldd, int nsm,
                    cudaStream_t st);
cudaError_t prepare_refine_kernels();
void launch_refine_core(const float* Ra1, const float* Ra2, const float* Rb1, const float* Rb2, int ld,
                        const double* C, int r, double* core, cudaStream_t st, const int* skip = nullptr);
// SVD of an n x n float64 matrix (n <= 64), leading r triplets, computed in float64 or,
// with f32, in float32 (one-sided Jacobi either way).
void launch_svd_small(const double* A, int n, int r, double* U, float* sigma, double* V, cudaStream_t st,
                      const int* skip = nullptr, bool f32 = false);

// GreBsmo (k_grebsmo.cu): the S-step's plan (one candidate pass at the key of lambda + 1
// ulp), the soft-threshold emit S = R - lambda sgn R over every candidate, column norms
// from a Gram, and a small float64 product of two r x r factors.
struct SoftEmitArgs {
  Ctl* ctl;
  const long long* cand_idx;
  const float* cand_val;
  unsigned long long cand_cap;
  long long s_cap;         // entries the S buffers hold
  long long* S_idx[2];
  float* S_val[2];
  unsigned* sbits;         // as in EmitArgs
  long long sbits_words;
  float lambda;
};
void launch_soft_plan(Ctl* ctl, unsigned guess, cudaStream_t st);
void launch_emit_soft(const SoftEmitArgs& a, int nsm, cudaStream_t st);
void launch_colnorm(const float* W, const double* g64, int64_t n, int RP, int r, float* Vh, float* sigma, int nsm,
                    cudaStream_t st, const int* skip = nullptr);
// out (r x r, float64) = A B (A, B float32, stride ld), transposed with trans, then row i
// scaled by rowscale[i] (nullable).
void launch_rmul(const float* A, const float* B, int ld, int r, double* out, int trans, const float* rowscale,
                 cudaStream_t st, const int* skip = nullptr);
// LinGoDec: out (d x r, float64) = T1 T2 Vr diag(sigma) (T1, T2 upper triangular d x d,
// stride ld; Vr d x r float64).
void launch_lingo_g(const float* T1, const float* T2, int ld, const double* Vr, const float* sigma, int d, int r,
                    double* out, cudaStream_t st);

// MSE training (k_mse.cu): gather of a label's rows of the residual plus its block, scatter
// back minus the new block, sparse axpy, the initial residual, X - R.
void launch_mse_gather(const float* R, int64_t ldr, const int64_t* rows, int64_t nrows, int64_t p, const float* X,
                       int64_t ldx, const float* invD, const float* U, int64_t ldu, const float* sigma, const float* V,
                       int64_t ldv, int r, float* N, int64_t ldn, int nsm, cudaStream_t st);
void launch_mse_scatter(float* R, int64_t ldr, const int64_t* rows, int64_t nrows, int64_t p, const float* N,
                        int64_t ldn, const float* U, int64_t ldu, const float* sigma, const float* V, int64_t ldv,
                        int r, int nsm, cudaStream_t st);
void launch_sparse_axpy(float* R, int64_t ldr, int64_t p, const int64_t* idx, const float* val, int64_t nnz,
                        float alpha, int nsm, cudaStream_t st);
void launch_mse_init(const float* X, int64_t ldx, const float* invD, int64_t rows, int64_t p, float* R, int64_t ldr,
                     int nsm, cudaStream_t st);
void launch_sub(const float* X, int64_t ldx, const float* R, int64_t ldr, int64_t rows, int64_t p, float* out,
                int64_t ldo, int nsm, cudaStream_t st);

// L (m x n, row stride ldl) = U diag(sigma) V^T, U m x r (ldu), V n x r (ldv) (k_dense.cu).
void launch_lowrank_dense(const float* U, int64_t ldu, const float* sigma, const float* V, int64_t ldv, int64_t m,
                          int64_t n, int r, float* L, int64_t ldl, cudaStream_t st);

// Small helpers.
void launch_fill_zero(void* p, size_t bytes, cudaStream_t st);
// dst (n x ldd) = src^T (src m x n with stride lds)
// dst = src^T, optionally times scale[0]
void launch_transpose(const float* src, int64_t m, int64_t n, int64_t lds, float* dst, int64_t ldd,
                      cudaStream_t st, const float* scale = nullptr);
void launch_pad_copy(const float* src, int64_t rows, int cols, int64_t lds, float* dst, int RP,
                     cudaStream_t st);
void launch_unpad_copy(const float* src, int64_t rows, int RP, float* dst, int cols,
                       cudaStream_t st);
// *out += sum of X^2 (float64 atomics: clear *out first for a fresh sum)
void launch_sumsq(const float* X, int64_t m, int64_t n, int64_t ldx, double* out, int nsm,
                  cudaStream_t st);
void launch_sort_coo(long long* idx, float* val, long long nnz, void* scratch, size_t scratch_bytes,
                     int idx_bits, cudaStream_t st);
size_t sort_coo_scratch(long long nnz);

}  // namespace godec
