// Shared device-side definitions of the GB300 quadric rasterizer (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qgs.h"

namespace qgs {

constexpr int TILE = 16;
constexpr int BLOCK = TILE * TILE;  // one thread per pixel of a tile
constexpr int NGRAD = 20;           // per-primitive gradient record (floats)
constexpr int NGRAD_PAD = 20;       // 80 B: 16-byte aligned records

// Per-primitive projected state: one 128-byte record (8 x float4), written by the
// preprocessing kernel for the visible primitives and gathered by the compositing
// kernels in sorted order (one cache line per primitive).
//   f[0] = (qa, 2qb, qc, 2la)     screen-space conic of the chord ellipsoid holding the
//   f[2].xy = (2lb, 0)              support: dx (qa dx + 2qb dy - 2la) + dy (qc dy - 2lb) <= 1
//                                   for the pixel offset (dx, dy) from the projected centre
//   f[1] = projected centre as double-float (pcx_hi, pcx_lo, pcy_hi, pcy_lo)
//   f[2].zw = (inv_z, z_mu)
//   f[3] = (W00, W10, W01, W11)   W = R_cw * R: camera-from-local rotation
//   f[4] = (W02, W12, g_x, g_y)   g = W^T mu_cam / z_mu: local direction of the centre ray
//   f[5] = (g_z, a, b, opacity)
//   f[6] = (1/s_u^2, 1/s_v^2, W20, W21)
//   f[7] = (W22, r, g, b)         colour from SH, clamped at 0
struct __align__(16) PrimState {
  float4 f[8];
};
static_assert(sizeof(PrimState) == 128, "PrimState must be one 128-byte line");

struct RasterParams {
  int W, H, tiles_x, tiles_y;
  float cx, cy, inv_fx, inv_fy;
  float near_plane;
  float alpha_max, alpha_min, T_min, grazing_eps;
  uint32_t id_mask;  // projected-state index = sorted id & id_mask (low bits of a packed key)
};

}  // namespace qgs
