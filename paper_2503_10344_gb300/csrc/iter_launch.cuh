// Launchers of the fused step kernels for one (iterate type, value type)
// pair; each iter_*.cu translation unit instantiates one pair.
#pragma once

#include <algorithm>

#include "internal.h"
#include "iter_kernels.cuh"
#include "tile_kernels.cuh"
#include "smem_kernels.cuh"
#include "wtile_kernels.cuh"

namespace pdlp {

template <typename T, typename V>
IterData<T, V> typed(const IterRaw& r) {
  IterData<T, V> d;
  d.a_ptr = r.a_ptr; d.a_col = r.a_col; d.a_val = (const V*)r.a_val;
  d.t_ptr = r.t_ptr; d.t_col = r.t_col; d.t_val = (const V*)r.t_val;
  d.a_long = r.a_long; d.t_long = r.t_long;
  d.a_nlong = r.a_nlong; d.t_nlong = r.t_nlong; d.a_thresh = r.a_thresh; d.t_thresh = r.t_thresh;
  d.m = r.m; d.n = r.n;
  d.c = (const T*)r.c; d.l = (const T*)r.l; d.u = (const T*)r.u; d.q = (const T*)r.q;
  d.tw = (const T*)r.tw; d.sw = (const T*)r.sw;
  d.row_kind = r.row_kind;
  for (int k = 0; k < 2; ++k) {
    d.x[k] = (vec2_t<T>*)r.x[k]; d.y[k] = (T*)r.y[k];
  }
  d.sum_x = (T*)r.sum_x; d.sum_y = (T*)r.sum_y;
  d.part_p = (T*)r.part_p; d.part_d = (T*)r.part_d;
  d.grid_p_short = r.grid_p_short; d.grid_p = r.grid_p;
  d.grid_d_short = r.grid_d_short; d.grid_d = r.grid_d;
  d.st = r.st;
  d.count = r.count;
  d.cond = r.cond;
  d.loop_cap = r.loop_cap;
  d.tp = r.tp;
  d.td = r.td;
  d.tile = r.tile;
  d.tt = r.tt;
  d.ta = r.ta;
  d.grid_tt = r.grid_tt;
  d.grid_ta = r.grid_ta;
  d.work_tt = r.work_tt;
  d.work_ta = r.work_ta;
  d.tslot = r.tslot;
  d.ord_t = r.ord_t;
  d.ord_a = r.ord_a;
  d.hx = (T*)r.hx;
  d.hy = (T*)r.hy;
  d.hax = (const T*)r.hax;
  d.hay = (const T*)r.hay;
  return d;
}

// The float32 primal kernel gathers y (4 bytes per row of A): ask for the
// largest L1 (the kernel uses almost no shared memory) so that y stays cached
// on the SM.  Set once per instantiation and device.
template <typename K>
cudaError_t prefer_l1(K kernel) {
  static int done_dev = -1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || done_dev == dev) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  if (e == cudaSuccess) done_dev = dev;
  return e;
}

template <int LANES, typename T, typename V, bool IMPLICIT, bool H>
cudaError_t launch_one(int which, const IterData<T, V>& d, cudaStream_t s) {
  if (which == IK_PRIMAL) {
    const cudaError_t e = prefer_l1(k_primal<LANES, T, V, IMPLICIT, H>);
    if (e != cudaSuccess) return e;
  }
  switch (which) {
    case IK_PRIMAL: return launch_pdl(k_primal<LANES, T, V, IMPLICIT, H>, d.grid_p, kBlock, s, d);
    case IK_DUAL: {  // the dual step, then the step decision of every LP
      const cudaError_t e = launch_pdl(k_dual<LANES, T, V, IMPLICIT, H>, d.grid_d, kBlock, s, d);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_decide<T, V>, d.count, kBlock, s, d);
    }
    default: return cudaErrorInvalidValue;
  }
}

// The tile kernel of one orientation: the staged block tiles (kTileStages stages of
// dynamic shared memory, allowed for the device by tile_resident during the setup)
// or the warp tiles.
template <typename V, bool IMPLICIT, bool DUAL>
cudaError_t launch_tile(const IterData<float, V>& d, cudaStream_t s) {
  const int grid = DUAL ? d.grid_ta : d.grid_tt;
  if (d.tile == 2) return launch_pdl(k_wtile<V, IMPLICIT, DUAL>, grid, kBlock, s, d);
  const int smem = kTileStages * StageLayout<V, DUAL>::bytes;
  return launch_pdl_smem(k_tile<V, IMPLICIT, DUAL>, grid, kBlock, smem, s, d);
}

// Blocks of the tile kernel (form 1 or 2) of one orientation that fit on the device at
// once; for form 1 also allows the kernel its dynamic shared memory on this device.
template <typename V, bool IMPLICIT, bool DUAL>
cudaError_t tile_resident(int form, int* blocks) {
  int per_sm = 0;
  cudaError_t e;
  if (form == 2) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wtile<V, IMPLICIT, DUAL>, kBlock, 0);
  } else {
    auto kern = k_tile<V, IMPLICIT, DUAL>;
    const int smem = kTileStages * StageLayout<V, DUAL>::bytes;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem);
  }
  if (e != cudaSuccess) return e;
  *blocks = std::max(1, per_sm) * device_sm_count();
  return cudaSuccess;
}

// H: the Halpern variant's step kernels (the tile forms have none)
template <typename T, typename V, bool IMPLICIT, bool H = false>
cudaError_t launch_iter_t(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  const IterData<T, V> d = typed<T, V>(r);
  if constexpr (std::is_same<T, float>::value && !H) {
    if (r.tile) {
      if (which == IK_PRIMAL) return launch_tile<V, IMPLICIT, false>(d, s);
      if (which != IK_DUAL) return cudaErrorInvalidValue;
      const cudaError_t e = launch_tile<V, IMPLICIT, true>(d, s);
      if (e != cudaSuccess) return e;
      return launch_pdl(k_decide<T, V>, d.count, kBlock, s, d);
    }
  }
  switch (lanes) {
    case 1: return launch_one<1, T, V, IMPLICIT, H>(which, d, s);
    case 2: return launch_one<2, T, V, IMPLICIT, H>(which, d, s);
    case 4: return launch_one<4, T, V, IMPLICIT, H>(which, d, s);
    case 8: return launch_one<8, T, V, IMPLICIT, H>(which, d, s);
    case 16: return launch_one<16, T, V, IMPLICIT, H>(which, d, s);
    case 32: return launch_one<32, T, V, IMPLICIT, H>(which, d, s);
    default: return cudaErrorInvalidValue;
  }
}

// Persistent attempts kernel (k_persist) of the lanes pair (LA over A, LT over
// A^T): one cooperative launch of `grid` blocks (0 = as many as can be resident,
// at most four per SM); *grid_out receives the grid used.
template <int LA, int LT, typename T, typename V, bool IMPLICIT>
cudaError_t launch_persist_one(const IterData<T, V>& d, int max_attempts, int grid,
                               int* grid_out, cudaStream_t s) {
  auto kern = k_persist<LA, LT, T, V, IMPLICIT>;
  if (grid <= 0) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    grid = std::min(per_sm, 4) * device_sm_count();
  }
  if (grid_out) *grid_out = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, d, max_attempts);
}

template <int LA, typename T, typename V, bool IMPLICIT>
cudaError_t launch_persist_la(int lanes_t, const IterData<T, V>& d, int max_attempts, int grid,
                              int* grid_out, cudaStream_t s) {
  switch (lanes_t) {
    case 2: return launch_persist_one<LA, 2, T, V, IMPLICIT>(d, max_attempts, grid, grid_out, s);
    case 4: return launch_persist_one<LA, 4, T, V, IMPLICIT>(d, max_attempts, grid, grid_out, s);
    case 8: return launch_persist_one<LA, 8, T, V, IMPLICIT>(d, max_attempts, grid, grid_out, s);
    case 16: return launch_persist_one<LA, 16, T, V, IMPLICIT>(d, max_attempts, grid, grid_out, s);
    case 32: return launch_persist_one<LA, 32, T, V, IMPLICIT>(d, max_attempts, grid, grid_out, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, typename V, bool IMPLICIT>
cudaError_t launch_persist_t(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                             int grid, int* grid_out, cudaStream_t s) {
  const IterData<T, V> d = typed<T, V>(r);
  if (grid == 1 && r.smem.bytes > 0) {
    // one block with the LP in shared memory (allowed its dynamic shared memory once
    // per device, at the setup's probe launch, outside any capture)
    auto kern = k_smem<T, V, IMPLICIT>;
    static int allowed_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (allowed_dev != dev) {
      int optin = 0;
      e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - kSmemStatic);
      if (e != cudaSuccess) return e;
      allowed_dev = dev;
    }
    if (grid_out) *grid_out = 1;
    kern<<<1, kBlock, r.smem.bytes, s>>>(d, r.smem, max_attempts);
    return cudaGetLastError();
  }
  switch (lanes_a) {
    case 2: return launch_persist_la<2, T, V, IMPLICIT>(lanes_t, d, max_attempts, grid, grid_out, s);
    case 4: return launch_persist_la<4, T, V, IMPLICIT>(lanes_t, d, max_attempts, grid, grid_out, s);
    case 8: return launch_persist_la<8, T, V, IMPLICIT>(lanes_t, d, max_attempts, grid, grid_out, s);
    case 16: return launch_persist_la<16, T, V, IMPLICIT>(lanes_t, d, max_attempts, grid, grid_out, s);
    case 32: return launch_persist_la<32, T, V, IMPLICIT>(lanes_t, d, max_attempts, grid, grid_out, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pdlp
