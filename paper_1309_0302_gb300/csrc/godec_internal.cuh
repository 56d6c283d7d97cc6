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

constexpr int kMaxRP = 64;          // maximum padded rank
constexpr int kHistBins = 4096;     // first radix digit: key bits 30..19
constexpr int kD1Shift = 19;
constexpr int kNumSelRounds = 7;    // 3 key digits + 4 index digits

// Pass modes of the residual (S-step) kernel.
enum PassMode : int { PASS_NONE = 0, PASS_FULL = 1, PASS_CAND = 2 };

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
  double m_logscale;            // M is stored divided by exp(m_logscale)
  // --- histograms ------------------------------------------------------------
  unsigned hist[kHistBins];     // digit-1 histogram of |R| keys (full pass)
  unsigned sel_hist[kHistBins];
};

// --------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All take the context stream.
// --------------------------------------------------------------------------------

// Split-K streaming product: part[s] (outdim x RP) = partial of Z B (trans=0,
// outdim = m, K = n) or Z^T C (trans=1, outdim = n, K = m) over K-split s.
// `Zh` may be bf16 (bf16 != 0) with the same layout and row stride.
struct PassArgs {
  const void* Z;
  int bf16;
  int64_t m, n, ldz;
  const float* B;        // K x RP
  float* part;           // splits x outdim x RP
  int splits;
  int64_t kchunk;        // K range per split (multiple of 32)
  int trans;
  int RP;
  const Ctl* ctl;        // nullable; abort flag checked
};
void launch_pass(const PassArgs& a, cudaStream_t st);
void pass_geometry(int64_t outdim, int64_t K, int nsm, int* splits, int64_t* kchunk);

// out (rows x RP) = sum_s part[s]; gram partials per 64-row block (RP x RP);
// gram_mode 0 = none, 1 = float32, 2 = float64 (exact products, double sums).
void launch_reduce(const float* part, int splits, int64_t rows, int RP, float* out,
                   void* gram_part, int gram_mode, const Ctl* ctl, cudaStream_t st);
int64_t reduce_blocks(int64_t rows);

// Q (rows x RP) = P (rows x RP) * T (RP x RP, upper triangular if upper != 0),
// optional float32 gram partials of Q.
void launch_apply(const float* P, int64_t rows, int RP, const float* T, int upper, float* Q,
                  float* gram_part, const Ctl* ctl, cudaStream_t st);

// One-block kernels on r x r matrices (see k_small.cu).
struct CholArgs {
  const void* gram_part;   // nblk x RP x RP partials (float or double)
  int gram_double;
  int64_t nblk;
  int r, RP;
  float* R;                // RP x RP upper triangular (out)
  float* Rinv;             // RP x RP (out)
  float* M;                // RP x RP: if accumulate, M := R * M (in/out)
  int accumulate;          // 0 none, 1 M := R*M, 2 M := R (start)
  int rank_test;           // run the pivoted rank test (needs gram_double)
  double rank_tol;
  Ctl* ctl;
};
void launch_chol(const CholArgs& a, cudaStream_t st);

struct SvdArgs {
  const float* M;          // RP x RP
  int r, RP, q;
  float* Um;               // RP x RP  (left vectors times sigma^(1/(2q+1)) NOT applied)
  float* Vm;               // RP x RP
  float* sigma;            // RP: sigma_L = s^(1/(2q+1)), descending, zero-padded
  Ctl* ctl;
};
void launch_svd_root(const SvdArgs& a, cudaStream_t st);

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
  void* Z16;               // nullable bf16 copy of Z (same ldz)
};
void launch_emit(const EmitArgs& a, int nsm, cudaStream_t st);
void launch_z_update(const EmitArgs& a, int nsm, cudaStream_t st);
// Reset the per-iteration S-step state (after an aborted iteration or at start).
void launch_reset_iter(Ctl* ctl, cudaStream_t st);

// Error text returned by godec_last_error(NULL) for calls without a context.
void set_static_error(const char* fmt, ...);

// Kernel attributes (dynamic shared memory limits); call before launching or capturing.
cudaError_t prepare_small_kernels();
cudaError_t prepare_select_kernels();

// Small helpers.
void launch_fill_zero(void* p, size_t bytes, cudaStream_t st);
void launch_pad_copy(const float* src, int64_t rows, int cols, int64_t lds, float* dst, int RP,
                     cudaStream_t st);
void launch_unpad_copy(const float* src, int64_t rows, int RP, float* dst, int cols,
                       cudaStream_t st);
void launch_sumsq(const float* X, int64_t m, int64_t n, int64_t ldx, double* out, int nsm,
                  cudaStream_t st);
void launch_sort_coo(long long* idx, float* val, long long nnz, void* scratch, size_t scratch_bytes,
                     int idx_bits, cudaStream_t st);
size_t sort_coo_scratch(long long nnz);

}  // namespace godec
