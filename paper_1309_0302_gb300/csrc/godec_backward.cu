// Differentiated form: reverse-mode gradient with respect to X of a loss of L_T after T
// unrolled iterations of Algorithm 1 at q = 0, with the supports of S_1 .. S_{T-1} frozen.
//
// At q = 0 the L-step is L = Y1 (A2^T Y1)^{-1} Y2^T = Z P, with A2 = Z A1, Y2 = Z^T A2 and
// P = Y2 (Y2^T Y2)^{-1} Y2^T the projector on range(Y2) (Sec. 3.1, eq. lr_app); with the
// support Omega_t frozen, S_t = M_t * (X - L_t) and Z_{t+1} = (1 - M_t) * X + M_t * L_t.
// Differentiating:  dL = dZ P + Z dP,  dP = (I - P) dY2 Y2^+ + (Y2^+)^T dY2^T (I - P),
// dY2 = dZ^T Z A1 + Z^T dZ A1.  For a gradient G of L_t, with W = (Y2^T Y2)^{-1} and
// Y2p = Y2 W = (Y2^+)^T:
//     a   = G Y2p,   b = G^T (Z Y2p),   gY2 = (I - P) (Z^T a + b),
//     gZ  = a Y2^T + (Z A1) gY2^T + (Z gY2) A1^T            (rank <= 3r),
// and Z_t routes gZ to X outside Omega_{t-1} and to L_{t-1} on it:
//     dX += (1 - M_{t-1}) * gZ_t,   G_{t-1} = M_{t-1} * gZ_t   (M_0 = 0).
//
// The forward sweep recomputes and checkpoints the per-iteration factors (A2, Y2, Y2p,
// Q, Z Y2p and L_t on Omega_t; Q an orthonormal basis of range(Y2) from CholeskyQR2);
// the backward sweep reuses Z_t and Z_t^T kept from the forward sweep when all T of them
// fit in a quarter of the free device memory, and otherwise rebuilds them from X and the
// checkpointed values.  Streaming products with Z_t and Z_t^T run on the tensor-core product kernel
// (float32 accuracy); the r x r solve is the Cholesky kernel of the L-step.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "godec.h"
#include "godec_internal.cuh"

namespace godec {
void launch_spmm(const int64_t* idx, const float* val, int64_t nnz, int64_t n, const float* B, int64_t ldb, int c,
                 int trans, float* out, int64_t ldo, cudaStream_t st);
void launch_eval_lr(const int64_t* idx, int64_t nnz, int64_t n, const float* U, int64_t ldu, const float* V,
                    int64_t ldv, int K, float* vals, float* D, int64_t ldd, cudaStream_t st);
void launch_scatter_set(const int64_t* idx, const float* vals, int64_t nnz, int64_t n, float* Z, int64_t ldz,
                        cudaStream_t st);
void launch_outer_acc(const float* U, int64_t ldu, const float* V, int64_t ldv, int K, int64_t m, int64_t n,
                      float beta, float* D, int64_t ldd, cudaStream_t st);
void launch_axpy(const float* x, float* y, int64_t count, float alpha, cudaStream_t st);
}  // namespace godec

namespace {

using namespace godec;

constexpr int kCrossParts = 256;

// Stream-ordered scratch of one call; freed (stream-ordered) on destruction.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  bool ok = true;
  template <typename T>
  T* get(size_t elems) {
    void* p = nullptr;
    if (!ok || cudaMallocAsync(&p, std::max<size_t>(elems, 1) * sizeof(T), st) != cudaSuccess) {
      ok = false;
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
};

// A float32 source of streaming products (Z_t, Z_t^T or a dense gradient and its
// transpose) with its tensor map, product geometry and power-of-two scale.
struct Source {
  alignas(64) unsigned char map[128];
  const float* p = nullptr;
  int64_t rows = 0, K = 0, ld = 0;
  TcGeom geom;
  float* zscale = nullptr;     // {s, 1/s} on the device
  unsigned* zmax = nullptr;
};

struct Engine {
  cudaStream_t st;
  int nsm = 0, RP = 0;
  int64_t ldb = 0;
  void* Bs = nullptr;                          // 2 RP x ldb halves (split transposed operand)
  alignas(64) unsigned char mapB[2][128];      // over Bs with K = n (index 0) and K = m (index 1)
  int64_t Kb[2] = {0, 0};
  float *Bp = nullptr, *cscale = nullptr, *part = nullptr, *Yp = nullptr;
  unsigned* cnt = nullptr;
  int* pend = nullptr;

  // Y (rows x c, dense) = src * B (K x c, dense rows of c)
  void mul(const Source& s, const float* B, int c, float* Y) {
    const int bi = (s.K == Kb[0]) ? 0 : 1;
    launch_pad_copy(B, s.K, c, c, Bp, RP, st);
    launch_split_t(Bp, s.K, RP, Bs, ldb, cscale, st);
    TcLaunch l{};
    l.mapA = s.map;
    l.mapB = mapB[bi];
    l.rows = s.rows;
    l.K = s.K;
    l.RP = RP;
    l.geom = s.geom;
    l.part = part;
    l.counters = cnt;
    l.out = Yp;
    l.cscale = cscale;
    l.zscale = s.zscale;
    l.pend = pend;
    launch_prod_tc(l, st);
    launch_unpad_copy(Yp, s.rows, RP, Y, c, st);
  }
};

bool setup_source(Source& s, const float* p, int64_t rows, int64_t K, int64_t ld, int nsm, float* zscale,
                  unsigned* zmax) {
  s.p = p;
  s.rows = rows;
  s.K = K;
  s.ld = ld;
  s.geom = tc_geometry(rows, K, nsm);
  s.zscale = zscale;
  s.zmax = zmax;
  return make_tmap_f32(s.map, p, rows, K, ld, 128);
}

}  // namespace

extern "C" godec_status godec_backward(const float* X, int64_t m, int64_t n, int64_t ldx, const float* A1, int32_t r,
                                       int32_t T, const int64_t* const* supports, const int64_t* support_nnz,
                                       const float* gU, const float* gV, int32_t g_rank, const float* gL, int64_t ldg,
                                       float* dX, int64_t lddx, int32_t flags, void* stream) {
  const bool lowrank = gU && gV;
  if (!X || !A1 || !dX || m < 1 || n < 1 || ldx < n || lddx < n || r < 1 || r > GODEC_MAX_RANK || r > m ||
      r > n || T < 1 || (T > 1 && (!supports || !support_nnz)) || lowrank == (gL != nullptr) ||
      (lowrank && (g_rank < 1 || g_rank > GODEC_MAX_RANK)) || (gL && ldg < n) || (ldx * 4) % 16 != 0 ||
      (gL && (ldg * 4) % 16 != 0) || (flags & ~GODEC_BACKWARD_REBUILD)) {
    set_static_error("godec_backward: invalid argument");
    return GODEC_ERR_ARG;
  }
  for (int t = 0; t + 1 < T; ++t)
    if (support_nnz[t] < 0 || support_nnz[t] > m * n || (support_nnz[t] > 0 && !supports[t])) {
      set_static_error("godec_backward: invalid support %d", t + 1);
      return GODEC_ERR_ARG;
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      prepare_tc_kernels() != cudaSuccess || prepare_small_kernels() != cudaSuccess) {
    set_static_error("godec_backward: no CUDA device");
    return GODEC_ERR_CUDA;
  }
  const int RP = (r + 7) / 8 * 8, R3 = 3 * r;
  const int64_t mx = std::max(m, n), ldz = (n + 63) / 64 * 64, ldzt = (m + 63) / 64 * 64;
  Scratch sc{st};
  // Iterates Z_t and Z_t^T: one copy each for all t, rebuilt in the backward sweep, or (when
  // all T of them fit in a quarter of the free device memory) one per t, kept from the
  // forward sweep, which saves the backward sweep's copy, scatter, transpose and scale.
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
  const bool keep = !(flags & GODEC_BACKWARD_REBUILD) &&
                    (double)T * (double)(m * ldz + n * ldzt) * sizeof(float) <= 0.25 * (double)free_b;
  const int nzb = keep ? T : 1;
  std::vector<float*> Zb(nzb), Ztb(nzb);
  for (int b = 0; b < nzb; ++b) {
    Zb[b] = sc.get<float>((size_t)m * ldz);
    Ztb[b] = sc.get<float>((size_t)n * ldzt);
  }
  float* Gt = gL ? sc.get<float>((size_t)n * ldzt) : nullptr;      // dense gradient transposed
  Engine E;
  E.st = st;
  E.nsm = nsm;
  E.RP = RP;
  E.ldb = (mx + 7) / 8 * 8;
  E.Bs = sc.get<unsigned short>((size_t)2 * RP * E.ldb);
  E.Bp = sc.get<float>((size_t)mx * RP);
  E.cscale = sc.get<float>(RP);
  E.Yp = sc.get<float>((size_t)mx * RP);
  float* zsc = sc.get<float>(2 * (size_t)nzb + 2);     // {s, 1/s} of each Z_t copy, then of the dense gradient
  unsigned* zmax = sc.get<unsigned>((size_t)nzb + 1);
  std::vector<Source> sZs(nzb), sZts(nzb);
  Source sG, sGt;
  // per-iteration checkpoints (forward sweep)
  std::vector<float*> A2(T), Y2(T), Y2p(T), Qk(T), ZY2p(T), Lv(T);
  for (int t = 0; t < T; ++t) {
    A2[t] = sc.get<float>((size_t)m * r);
    Y2[t] = sc.get<float>((size_t)n * r);
    Y2p[t] = sc.get<float>((size_t)n * r);
    Qk[t] = sc.get<float>((size_t)n * r);
    ZY2p[t] = sc.get<float>((size_t)m * r);
    Lv[t] = (t + 1 < T && support_nnz[t] > 0) ? sc.get<float>((size_t)support_nnz[t]) : nullptr;
  }
  int64_t kmax = 0;
  for (int t = 0; t + 1 < T; ++t) kmax = std::max(kmax, support_nnz[t]);
  float* gv = sc.get<float>((size_t)std::max<int64_t>(kmax, 1));   // G_{t-1} on Omega_{t-1}
  float* Y2T = sc.get<float>((size_t)n * r);
  float* a = sc.get<float>((size_t)m * r);
  float* Wn = sc.get<float>((size_t)n * r);
  float* Zg = sc.get<float>((size_t)m * r);
  float* Uf = sc.get<float>((size_t)m * R3);
  float* Vf = sc.get<float>((size_t)n * R3);
  float* Rm = sc.get<float>((size_t)RP * RP * 4);                  // R1, T1, R2, T2 of CholeskyQR2
  double* g64 = sc.get<double>((size_t)RP * RP);
  double* Msm = sc.get<double>((size_t)GODEC_MAX_RANK * GODEC_MAX_RANK);
  double* cpart = sc.get<double>((size_t)kCrossParts * GODEC_MAX_RANK * GODEC_MAX_RANK);
  Ctl* ctl = sc.get<Ctl>(1);
  if (sc.ok) {
    const TcGeom gz = tc_geometry(m, n, nsm), gzt = tc_geometry(n, m, nsm);
    size_t npart = 0, npend = 0;
    int64_t tiles = 0;
    for (const TcGeom& g : {gz, gzt}) {
      npart = std::max(npart, (size_t)g.tiles * g.maxseg * 128 * RP);
      npend = std::max(npend, (size_t)g.G * g.maxpend);
      tiles = std::max(tiles, g.tiles);
    }
    E.part = sc.get<float>(npart);
    E.pend = sc.get<int>(npend);
    E.cnt = sc.get<unsigned>((size_t)tiles);
  }
  if (!sc.ok) {
    set_static_error("godec_backward: out of device memory");
    return GODEC_ERR_OOM;
  }
  cudaMemsetAsync(E.cnt, 0, (size_t)std::max(tc_geometry(m, n, nsm).tiles, tc_geometry(n, m, nsm).tiles) * sizeof(unsigned), st);
  cudaMemsetAsync(ctl, 0, sizeof(Ctl), st);
  E.Kb[0] = n;
  E.Kb[1] = m;
  bool mapped = make_tmap_f16(E.mapB[0], E.Bs, 2 * RP, n, E.ldb, 2 * RP) &&
                make_tmap_f16(E.mapB[1], E.Bs, 2 * RP, m, E.ldb, 2 * RP);
  for (int b = 0; b < nzb; ++b)
    mapped = mapped && setup_source(sZs[b], Zb[b], m, n, ldz, nsm, zsc + 2 * b, zmax + b) &&
             setup_source(sZts[b], Ztb[b], n, m, ldzt, nsm, zsc + 2 * b, zmax + b);
  if (gL) {
    mapped = mapped && setup_source(sG, gL, m, n, ldg, nsm, zsc + 2 * nzb, zmax + nzb) &&
             setup_source(sGt, Gt, n, m, ldzt, nsm, zsc + 2 * nzb, zmax + nzb);
  }
  if (!mapped) {
    set_static_error("godec_backward: tensor map encoding failed");
    return GODEC_ERR_CUDA;
  }
  const size_t rowb = sizeof(float);
  // Z_t = X with L_{t-1} on Omega_{t-1}; Z_t^T; the shared scale of both (copy slot b)
  auto build_Z = [&](int t) {
    const int b = keep ? t : 0;
    float *Z = Zb[b], *Zt = Ztb[b];
    cudaMemcpy2DAsync(Z, ldz * rowb, X, ldx * rowb, n * rowb, m, cudaMemcpyDeviceToDevice, st);
    if (t > 0 && support_nnz[t - 1] > 0) launch_scatter_set(supports[t - 1], Lv[t - 1], support_nnz[t - 1], n, Z, ldz, st);
    launch_transpose(Z, m, n, ldz, Zt, ldzt, st);
    launch_zscale(Z, m, n, ldz, zmax + b, zsc + 2 * b, nsm, st);
  };
  // ---------------- forward sweep: checkpoints ----------------
  for (int t = 0; t < T; ++t) {
    build_Z(t);
    const Source& sZ = sZs[keep ? t : 0];
    const Source& sZt = sZts[keep ? t : 0];
    E.mul(sZ, A1, r, A2[t]);                                   // A2 = Z A1
    E.mul(sZt, A2[t], r, Y2[t]);                               // Y2 = Z^T A2
    // Y2 = Q R by CholeskyQR2 (R = R2 R1), so that W = (Y2^T Y2)^{-1} = R^{-1} R^{-T} and
    // Y2p = Y2 W = Q T2^T T1^T are formed without squaring Y2's condition number
    const size_t rr = (size_t)RP * RP;
    float *R1 = Rm, *T1 = Rm + rr, *R2 = Rm + 2 * rr, *T2 = Rm + 3 * rr;
    launch_cross_gram(Y2[t], r, r, Y2[t], r, r, n, cpart, kCrossParts, g64, RP, st);
    launch_chol(g64, r, RP, R1, T1, ctl, st, 0.f);
    launch_tall_small_f(Y2[t], r, r, T1, RP, 0, r, n, 1.f, 0.f, Y2T, r, st);      // Q1 = Y2 T1
    launch_cross_gram(Y2T, r, r, Y2T, r, r, n, cpart, kCrossParts, g64, RP, st);
    launch_chol(g64, r, RP, R2, T2, ctl, st, 0.f);
    launch_tall_small_f(Y2T, r, r, T2, RP, 0, r, n, 1.f, 0.f, Qk[t], r, st);       // Q = Q1 T2
    launch_tall_small_f(Qk[t], r, r, T2, RP, 1, r, n, 1.f, 0.f, Y2T, r, st);       // Q T2^T
    launch_tall_small_f(Y2T, r, r, T1, RP, 1, r, n, 1.f, 0.f, Y2p[t], r, st);      // ... T1^T
    E.mul(sZ, Y2p[t], r, ZY2p[t]);                             // Y1 W = Z Y2p
    if (t + 1 < T && support_nnz[t] > 0)                       // L_t on Omega_t
      launch_eval_lr(supports[t], support_nnz[t], n, ZY2p[t], r, Y2[t], r, r, Lv[t], nullptr, 0, st);
  }
  // ---------------- backward sweep ----------------
  if (gL) {
    launch_transpose(gL, m, n, ldg, Gt, ldzt, st);
    launch_zscale(gL, m, n, ldg, zmax + nzb, zsc + 2 * nzb, nsm, st);
  }
  for (int t = T - 1; t >= 0; --t) {
    if (!keep) build_Z(t);
    const Source& sZ = sZs[keep ? t : 0];
    const Source& sZt = sZts[keep ? t : 0];
    // a = G Y2p and Wn = b = G^T (Z Y2p)
    if (t == T - 1 && gL) {
      E.mul(sG, Y2p[t], r, a);
      E.mul(sGt, ZY2p[t], r, Wn);
    } else if (t == T - 1) {
      launch_cross_gram(gV, g_rank, g_rank, Y2p[t], r, r, n, cpart, kCrossParts, Msm, r, st);
      launch_tall_small_d(gU, g_rank, g_rank, Msm, r, 0, r, m, 1.f, 0.f, a, r, st);
      launch_cross_gram(gU, g_rank, g_rank, ZY2p[t], r, r, m, cpart, kCrossParts, Msm, r, st);
      launch_tall_small_d(gV, g_rank, g_rank, Msm, r, 0, r, n, 1.f, 0.f, Wn, r, st);
    } else {
      cudaMemsetAsync(a, 0, (size_t)m * r * sizeof(float), st);
      cudaMemsetAsync(Wn, 0, (size_t)n * r * sizeof(float), st);
      launch_spmm(supports[t], gv, support_nnz[t], n, Y2p[t], r, r, 0, a, r, st);
      launch_spmm(supports[t], gv, support_nnz[t], n, ZY2p[t], r, r, 1, Wn, r, st);
    }
    // Wn += Z^T a;  gY2 = (I - P) Wn = Wn - Y2p (Y2^T Wn)
    E.mul(sZt, a, r, Y2T);
    launch_axpy(Y2T, Wn, (int64_t)n * r, 1.f, st);
    launch_cross_gram(Qk[t], r, r, Wn, r, r, n, cpart, kCrossParts, Msm, r, st);
    launch_tall_small_d(Qk[t], r, r, Msm, r, 0, r, n, -1.f, 1.f, Wn, r, st);     // Wn = (I - Q Q^T) Wn = gY2
    E.mul(sZ, Wn, r, Zg);                                       // Z gY2
    // factors of gZ_t: [a | A2 | Z gY2] [Y2 | gY2 | A1]^T
    cudaMemcpy2DAsync(Uf, R3 * rowb, a, r * rowb, r * rowb, m, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(Uf + r, R3 * rowb, A2[t], r * rowb, r * rowb, m, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(Uf + 2 * r, R3 * rowb, Zg, r * rowb, r * rowb, m, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(Vf, R3 * rowb, Y2[t], r * rowb, r * rowb, n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(Vf + r, R3 * rowb, Wn, r * rowb, r * rowb, n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpy2DAsync(Vf + 2 * r, R3 * rowb, A1, r * rowb, r * rowb, n, cudaMemcpyDeviceToDevice, st);
    launch_outer_acc(Uf, R3, Vf, R3, R3, m, n, t == T - 1 ? 0.f : 1.f, dX, lddx, st);
    // on Omega_{t-1}: gZ_t goes to L_{t-1} (next G) instead of X
    if (t > 0 && support_nnz[t - 1] > 0)
      launch_eval_lr(supports[t - 1], support_nnz[t - 1], n, Uf, R3, Vf, R3, R3, gv, dX, lddx, st);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_static_error("godec_backward: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  return GODEC_OK;
}
