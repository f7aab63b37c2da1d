// rd_sz_dev.cuh -- SZ point and block computations shared by the SZ passes,
// the fused batched estimate and the inspector (Sections "Prediction-Based
// Transformation" and "Estimation Based on Static Quantization").
#pragma once

#include <stdint.h>

#include "rd_device.cuh"

namespace rdk {

constexpr int kSzThreads = 256;

struct Nbr {
  // the 2^D corner values of the Lorenzo cell ending at a point; index bit k
  // set = one step back along axis D-1-k (bit 0 = fastest axis)
  float v[8];
};

template <int D>
__device__ __forceinline__ Nbr gather_cell(const FieldDev& f, const int* g) {
  Nbr c;
  constexpr int NC = 1 << D;
#pragma unroll
  for (int m = 0; m < NC; m++) {
    long long idx = 0;
    bool inside = true;
#pragma unroll
    for (int k = 0; k < D; k++) {
      int back = (m >> (D - 1 - k)) & 1;
      int gk = g[k] - back;
      inside = inside && gk >= 0;
      idx = idx * f.n[k] + gk;
    }
    c.v[m] = inside ? __ldg(f.x + idx) : 0.0f;
  }
  return c;
}

// x - Lorenzo(x) as nested float32 differences, last axis first:
//   1D: v0 - v1
//   2D: (v00 - v01) - (v10 - v11)
//   3D: 2D form on the current plane minus the 2D form on the plane behind.
template <int D>
__device__ __forceinline__ float est_residual(const Nbr& c) {
  if constexpr (D == 1) {
    return __fsub_rn(c.v[0], c.v[1]);
  } else if constexpr (D == 2) {
    return __fsub_rn(__fsub_rn(c.v[0], c.v[1]), __fsub_rn(c.v[2], c.v[3]));
  } else {
    float p0 = __fsub_rn(__fsub_rn(c.v[0], c.v[1]), __fsub_rn(c.v[2], c.v[3]));
    float p1 = __fsub_rn(__fsub_rn(c.v[4], c.v[5]), __fsub_rn(c.v[6], c.v[7]));
    return __fsub_rn(p0, p1);
  }
}

__device__ __forceinline__ int est_symbol(float r, float inv, int R) {
  float q = rintf(__fmul_rn(r, inv));
  return fabsf(q) < (float)R ? (int)q + kCenter : 0;
}

// Integer Lorenzo residual of the prequantised codes: sum over the cell's
// corners of (-1)^(steps back) Q.
template <int D>
__device__ __forceinline__ int gt_residual(const Nbr& c, float inv) {
  int r = 0;
#pragma unroll
  for (int m = 0; m < (1 << D); m++) {
    int q = __float2int_rn(__fmul_rn(c.v[m], inv));
    r += (__popc(m) & 1) ? -q : q;
  }
  return r;
}

template <int D>
__device__ __forceinline__ void point_coords(const FieldDev& f, long long u, int* g) {
  long long r = u;
#pragma unroll
  for (int k = D - 1; k >= 0; k--) {
    g[k] = (int)(r % f.n[k]);
    r /= f.n[k];
  }
}

template <int D>
__device__ __forceinline__ bool in_sampled_block(const FieldDev& f, const int* g) {
  bool s = true;
#pragma unroll
  for (int k = 0; k < D; k++) s = s && (((g[k] >> 2) % f.s[k]) == 0);
  return s;
}

// ---------------------------------------------------------------------------
// Estimator over the points of sampled blocks only: one thread per sampled
// block.  The thread reads the block with its one-cell halo on the low side
// ((4+1)^d values, zero outside the domain), a plane at a time: the 2D
// nested difference of each of the 16 points of a plane, minus that of the
// plane behind, is the 3D residual, in the same float32 operations and
// order as est_residual.
// ---------------------------------------------------------------------------
// Row y of plane z, values x0-1 .. x0+3 (zero outside the domain; values past
// the far edges feed no valid point and read as zero).
__device__ __forceinline__ void load_halo_row(const FieldDev& f, long long row, bool row_ok, int x0,
                                              int nx, float* v) {
  if (!row_ok) {
#pragma unroll
    for (int k = 0; k < 5; k++) v[k] = 0.0f;
    return;
  }
  const float* __restrict__ p = f.x + row * nx;
  v[0] = x0 > 0 ? __ldg(p + x0 - 1) : 0.0f;
  if (f.vec_ok && x0 + 4 <= nx) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p + x0));
    v[1] = q.x;
    v[2] = q.y;
    v[3] = q.z;
    v[4] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; k++) v[k + 1] = x0 + k < nx ? __ldg(p + x0 + k) : 0.0f;
  }
}

// Lattice index of a sampled block -> its first point per axis.
template <int D>
__device__ __forceinline__ void sampled_block_origin(const FieldDev& f, long long sb, int* o) {
  long long r = sb;
#pragma unroll
  for (int k = D - 1; k >= 0; k--) {
    const int l = (int)(r % f.L[k]);
    r /= f.L[k];
    o[k] = 4 * l * f.s[k];
  }
}

// res(r) receives the residual of every valid point of the block; for 3D
// blocks round_end() runs after each of the four planes, in every thread of
// the CTA (active or not).
template <int D, class Res, class RoundEnd>
__device__ __forceinline__ void sz_block_residuals(const FieldDev& f, long long sb, bool active,
                                                   Res&& res, RoundEnd&& round_end) {
  int o[3] = {0, 0, 0};
  if (active) sampled_block_origin<D>(f, sb, o);
  if constexpr (D == 1) {
    float v[5];
    load_halo_row(f, 0, active, o[0], f.n[0], v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool ok = active && o[0] + k < f.n[0];
      if (ok) res(__fsub_rn(v[k + 1], v[k]));
    }
  } else {
    const int ny = f.n[D - 2], nx = f.n[D - 1];
    const int y0 = o[D - 2], x0 = o[D - 1];
    // 2D nested differences of the 16 points of plane z (rows y0-1 .. y0+3)
    auto plane = [&](int z, bool z_ok, float* d2) {
      float v[5][5];
#pragma unroll
      for (int r = 0; r < 5; r++) {
        const int y = y0 - 1 + r;
        const bool ok = z_ok && y >= 0 && y < ny;
        const long long row = (D == 3 ? (long long)z * ny : 0ll) + y;
        load_halo_row(f, row, ok, x0, nx, v[r]);
      }
#pragma unroll
      for (int j = 0; j < 4; j++)
#pragma unroll
        for (int k = 0; k < 4; k++)
          d2[4 * j + k] = __fsub_rn(__fsub_rn(v[j + 1][k + 1], v[j + 1][k]),
                                    __fsub_rn(v[j][k + 1], v[j][k]));
    };
    float prev[16];
    const int nz = D == 3 ? f.n[0] : 1;
    const int z0 = D == 3 ? o[0] : 0;
    if (D == 3) plane(z0 - 1, active && z0 > 0, prev);
#pragma unroll 1
    for (int i = 0; i < (D == 3 ? 4 : 1); i++) {
      const int z = z0 + i;
      const bool z_ok = active && z < nz;
      float cur[16];
      plane(z, z_ok, cur);
#pragma unroll
      for (int t = 0; t < 16; t++) {
        const int j = t >> 2, k = t & 3;
        const bool ok = z_ok && y0 + j < ny && x0 + k < nx;
        const float r = D == 3 ? __fsub_rn(cur[t], prev[t]) : cur[t];
        if (ok) res(r);
      }
      if (D == 3) {
#pragma unroll
        for (int t = 0; t < 16; t++) prev[t] = cur[t];
        round_end();
      }
    }
  }
}

// Rows of four points per sampled block: 16 in 3D (plane i = t >> 2, row
// j = t & 3), 4 in 2D, 1 in 1D.
template <int D>
__host__ __device__ constexpr int est_rows() { return D == 3 ? 16 : D == 2 ? 4 : 1; }

// res(r) receives the residual of every valid point of row t of sampled
// block sb: the same nested first differences as sz_block_residuals, from
// the row itself, the row before it (y - 1) and, in 3D, those two rows of
// plane z - 1 (zero outside the domain), so one thread's loads are
// independent of each other.
template <int D, class Res>
__device__ __forceinline__ void sz_row_residuals(const FieldDev& f, long long sb, int t, bool active,
                                                 Res&& res) {
  int o[3] = {0, 0, 0};
  if (active) sampled_block_origin<D>(f, sb, o);
  if constexpr (D == 1) {
    float v[5];
    load_halo_row(f, 0, active, o[0], f.n[0], v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool ok = active && o[0] + k < f.n[0];
      if (ok) res(__fsub_rn(v[k + 1], v[k]));
    }
  } else {
    const int ny = f.n[D - 2], nx = f.n[D - 1];
    const int j = t & 3;
    const int y = o[D - 2] + j, x0 = o[D - 1];
    const int nz = D == 3 ? f.n[0] : 1;
    const int z = D == 3 ? o[0] + (t >> 2) : 0;
    const bool z_ok = active && z < nz;
    auto row_of = [&](int zz, int yy) { return (D == 3 ? (long long)zz * ny : 0ll) + yy; };
    float v11[5], v10[5];
    load_halo_row(f, row_of(z, y), z_ok && y < ny, x0, nx, v11);
    load_halo_row(f, row_of(z, y - 1), z_ok && y >= 1 && y - 1 < ny, x0, nx, v10);
    float v01[5], v00[5];
    if (D == 3) {
      const bool p_ok = active && z >= 1 && z - 1 < nz;
      load_halo_row(f, row_of(z - 1, y), p_ok && y < ny, x0, nx, v01);
      load_halo_row(f, row_of(z - 1, y - 1), p_ok && y >= 1 && y - 1 < ny, x0, nx, v00);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool ok = z_ok && y < ny && x0 + k < nx;
      const float cur = __fsub_rn(__fsub_rn(v11[k + 1], v11[k]), __fsub_rn(v10[k + 1], v10[k]));
      float r = cur;
      if (D == 3)
        r = __fsub_rn(cur, __fsub_rn(__fsub_rn(v01[k + 1], v01[k]), __fsub_rn(v00[k + 1], v00[k])));
      if (ok) res(r);
    }
  }
}

// add(sym) counts the linear code of every valid point of the block.
template <int D, class Add, class RoundEnd>
__device__ __forceinline__ void sz_est_block(const FieldDev& f, long long sb, bool active, float inv,
                                             int R, Add&& add, RoundEnd&& round_end) {
  sz_block_residuals<D>(f, sb, active, [&](float r) { add(est_symbol(r, inv, R)); }, round_end);
}

// add(sym) counts the linear code of every valid point of row t of block sb.
template <int D, class Add>
__device__ __forceinline__ void sz_est_row(const FieldDev& f, long long sb, int t, bool active,
                                           float inv, int R, Add&& add) {
  sz_row_residuals<D>(f, sb, t, active, [&](float r) { add(est_symbol(r, inv, R)); });
}

}  // namespace rdk
