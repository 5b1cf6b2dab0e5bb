// Launchers of the fused step kernels for one (iterate type, value type)
// pair; each iter_*.cu translation unit instantiates one pair.
#pragma once

#include "internal.h"
#include "iter_kernels.cuh"

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
  d.tp = r.tp;
  d.td = r.td;
  return d;
}

template <int LANES, typename T, typename V, bool IMPLICIT>
cudaError_t launch_one(int which, const IterData<T, V>& d, cudaStream_t s) {
  switch (which) {
    case IK_PRIMAL: k_primal<LANES, T, V, IMPLICIT><<<d.grid_p, kBlock, 0, s>>>(d); break;
    case IK_DUAL: k_dual<LANES, T, V, IMPLICIT><<<d.grid_d, kBlock, 0, s>>>(d); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, typename V, bool IMPLICIT>
cudaError_t launch_iter_t(int which, int lanes, const IterRaw& r, cudaStream_t s) {
  const IterData<T, V> d = typed<T, V>(r);
  switch (lanes) {
    case 2: return launch_one<2, T, V, IMPLICIT>(which, d, s);
    case 4: return launch_one<4, T, V, IMPLICIT>(which, d, s);
    case 8: return launch_one<8, T, V, IMPLICIT>(which, d, s);
    case 16: return launch_one<16, T, V, IMPLICIT>(which, d, s);
    case 32: return launch_one<32, T, V, IMPLICIT>(which, d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pdlp
