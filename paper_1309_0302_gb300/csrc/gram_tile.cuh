// Gram partial Y^T Y of one 128-row tile held in shared memory, shared by the tile
// completion of the streaming product and the stand-alone Gram kernel.
#pragma once

#include "godec_internal.cuh"

namespace godec {

// Ps: the tile's rows (up to 128, rows past the matrix zero), row stride ld floats.  Run by
// nthr threads (u = 0 .. nthr-1, whole warps).  The upper triangle in 4 x 4 blocks, each
// block's rows split over four adjacent lanes (row r to lane r mod 4), reduced by shuffles
// and mirrored on writing.  mode 1: float products summed in float, written as float;
// mode 2: exact float products (the fma residual kept) summed in double-float, written as
// double.  out: the tile's RP x RP partial.
__device__ __forceinline__ void gram_tile(const float* Ps, int ld, int RP, int mode, void* out, int u, int nthr) {
  constexpr int kRows = 128;
  const int nb = RP / 4, nblk = nb * (nb + 1) / 2, nit = nblk * 4;
  const int lane = u & 31;
  for (int base = u - lane; base < nit; base += nthr) {
    const int it = base + lane;
    const bool act = it < nit;
    const int blk = act ? it >> 2 : 0, sp = it & 3;
    int bi = 0, rem = blk;
    while (rem >= nb - bi) {
      rem -= nb - bi;
      ++bi;
    }
    const int bj = bi + rem;
    const float* pi = Ps + 4 * bi;
    const float* pj = Ps + 4 * bj;
    const bool wr = act && sp == 0;
    if (mode == 1) {
      float acc[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[e] = 0.f;
      if (act)
#pragma unroll 4
        for (int r = sp; r < kRows; r += 4) {
          const float* pr = pi + r * ld;
          const float* qr = pj + r * ld;
          const float uu[4] = {pr[0], pr[1], pr[2], pr[3]}, vv[4] = {qr[0], qr[1], qr[2], qr[3]};
#pragma unroll
          for (int i4 = 0; i4 < 4; ++i4)
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) acc[i4 * 4 + j4] = fmaf(uu[i4], vv[j4], acc[i4 * 4 + j4]);
        }
      float* gp = reinterpret_cast<float*>(out);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        float v = acc[e];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (wr) {
          const int i = 4 * bi + e / 4, j = 4 * bj + e % 4;
          gp[i * RP + j] = v;
          gp[j * RP + i] = v;
        }
      }
    } else {
      float hi[16], lo[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) hi[e] = lo[e] = 0.f;
      if (act)
#pragma unroll 1
        for (int r = sp; r < kRows; r += 4) {
          const float* pr = pi + r * ld;
          const float* qr = pj + r * ld;
          const float uu[4] = {pr[0], pr[1], pr[2], pr[3]}, vv[4] = {qr[0], qr[1], qr[2], qr[3]};
#pragma unroll
          for (int i4 = 0; i4 < 4; ++i4)
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) {
              const int e = i4 * 4 + j4;
              const float x = uu[i4], z = vv[j4];
              const float p = x * z, pe = fmaf(x, z, -p);
              const float sum = hi[e] + p, bb = sum - hi[e];
              lo[e] += ((hi[e] - (sum - bb)) + (p - bb)) + pe;
              hi[e] = sum;
            }
        }
      double* gp = reinterpret_cast<double*>(out);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        double d = (double)hi[e] + (double)lo[e];
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
        if (wr) {
          const int i = 4 * bi + e / 4, j = 4 * bj + e % 4;
          gp[i * RP + j] = d;
          gp[j * RP + i] = d;
        }
      }
    }
  }
}

}  // namespace godec
