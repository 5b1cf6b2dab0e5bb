// Fused PDHG step kernels (rows A4-A7 of the hot path).
//
// One step attempt is two launches:
//   k_primal  -- row-split CSR SpMV over A^T (one group of LANES lanes per
//                column), fused with the projected primal update
//                x' = proj_[l,u](x - tau (c - K^T y)) and the partial sums of
//                ||x' - x||^2 (scaled norm).
//   k_dual    -- row-split CSR SpMV over A, fused with the extrapolated dual
//                update y' = proj_Y(y + sigma (q - K(2x' - x))) and the partial
//                sums of ||y' - y||^2 and (y' - y)^T K (x' - x); its last block
//                reduces the partials in a fixed order and takes the adaptive
//                step-size decision (accept / retry) on the device.
// The primal iterate is stored as interleaved pairs (x'_j, x'_j - x_j): one
// vector gather per nonzero gives the dual kernel both K x' and K (x' - x),
// so K(2x' - x) = K x' + K dx and the step-size interaction term dy^T K dx are
// formed from K dx itself, not from the cancelling difference K x' - K x.
// Rows longer than a threshold are handled by extra blocks at the end of the
// grid, one block per long row, so a skewed row cannot stall a group.
//
// Two storage forms (both are the same preconditioned iteration):
//   IMPLICIT = false: K~ = D_r K D_c is stored; vectors live in scaled space.
//   IMPLICIT = true : the unscaled K is stored (bfloat16 or a bare pattern) and
//                     the scaling is folded into per-element steps
//                     tau_j = tau D_c,j^2 (tw), sigma_i = sigma D_r,i^2 (sw);
//                     the scaled norms divide by tw / sw.
#pragma once

#include "common.cuh"

namespace pdlp {

__device__ __forceinline__ float clampv(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }
__device__ __forceinline__ double clampv(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }
__device__ __forceinline__ float maxv(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double maxv(double a, double b) { return fmax(a, b); }

template <typename T, typename V>
struct IterData {
  const int* a_ptr; const int* a_col; const V* a_val;  // A (m rows)
  const int* t_ptr; const int* t_col; const V* t_val;  // A^T (n rows)
  const int* a_long; const int* t_long;                // rows handled by one block each
  int a_nlong, t_nlong, a_thresh, t_thresh;
  int m, n;
  const T* c; const T* l; const T* u; const T* q;      // iteration-space problem vectors
  const T* tw; const T* sw;                            // IMPLICIT step weights (else unused)
  const unsigned char* row_kind;                       // 1 = equality row (free dual)
  vec2_t<T>* x[2];                                     // (x_j, x_j - previous x_j) pairs
  T* y[2];
  T* sum_x; T* sum_y;
  double* part_p;                                      // [grid_p]
  double* part_d;                                      // [2][grid_d]
  int grid_p_short, grid_p, grid_d_short, grid_d;
  DevState* st;
};

// Rows r = g, g + G, ... of a CSR matrix, one aligned group of LANES lanes per
// row; rows longer than `thresh` are skipped here (the long-row blocks own them).
template <int LANES, typename Acc, typename Load, typename Epi>
__device__ __forceinline__ void rows_short(int nrows, const int* __restrict__ ptr, int thresh,
                                           int nblocks, Load load, Epi epi) {
  const int lane = threadIdx.x & (LANES - 1);
  const long long G = (long long)nblocks * kBlock / LANES;
  for (long long r = ((long long)blockIdx.x * kBlock + threadIdx.x) / LANES; r < nrows; r += G) {
    const int s = __ldg(ptr + r), e = __ldg(ptr + r + 1);
    if (e - s > thresh) continue;  // uniform within the group
    Acc acc{};
    for (int p = s + lane; p < e; p += LANES) acc += load(p);
    acc = group_sum<LANES>(acc);
    if (lane == 0) epi((int)r, acc);
  }
}

template <typename Acc>
__device__ __forceinline__ Acc block_allsum(Acc v) {
  __shared__ Acc sh[kWarps];
  v = group_sum<32>(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  Acc s{};
  if (threadIdx.x == 0)
    for (int i = 0; i < kWarps; ++i) s += sh[i];
  __syncthreads();
  return s;  // valid in thread 0
}

// Long rows: one block per row of the list, blocks [first, gridDim.x).
template <typename Acc, typename Load, typename Epi>
__device__ __forceinline__ void rows_long(const int* __restrict__ ptr, const int* __restrict__ list,
                                          int nlist, int first, Load load, Epi epi) {
  for (int k = blockIdx.x - first; k < nlist; k += gridDim.x - first) {
    const int r = list[k];
    const int s = ptr[r], e = ptr[r + 1];
    Acc acc{};
    for (int p = s + threadIdx.x; p < e; p += kBlock) acc += load(p);
    acc = block_allsum(acc);
    if (threadIdx.x == 0) epi(r, acc);
  }
}

template <typename T, typename V, int LANES, typename Epi, typename Vec>
__device__ __forceinline__ void spmv_rows(int nrows, const int* ptr, const int* col, const V* val,
                                          const Vec* vec, int thresh, const int* list, int nlist,
                                          int nshort, Epi epi) {
  auto load = [&](int p) -> T { return Ld<T, V>::get(val, p) * (T)__ldg(vec + __ldg(col + p)); };
  if ((int)blockIdx.x < nshort)
    rows_short<LANES, T>(nrows, ptr, thresh, nshort, load, epi);
  else
    rows_long<T>(ptr, list, nlist, nshort, load, epi);
}

// ---------------------------------------------------------------- A4: primal
template <int LANES, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_primal(IterData<T, V> d) {
  DevState* st = d.st;
  if (st->status != 0 || st->check_due) return;
  const int cur = st->cur;
  const vec2_t<T>* __restrict__ x = d.x[cur];
  vec2_t<T>* __restrict__ xn = d.x[cur ^ 1];
  const T* __restrict__ y = d.y[cur];
  const T tau = (T)(st->eta / st->omega);
  const double pw64 = st->pending_w;
  const T pw = (T)pw64;
  T dx2 = 0;
  auto epi = [&](int j, T aty) {
    const T xo = x[j].x;
    const T g = d.c[j] - aty;
    const T step = IMPLICIT ? tau * d.tw[j] : tau;
    const T xv = clampv(xo - step * g, d.l[j], d.u[j]);
    const T dd = xv - xo;
    vec2_t<T> o;
    o.x = xv;
    o.y = dd;
    xn[j] = o;
    if (pw64 != 0.0) d.sum_x[j] += pw * xo;  // A7: add the iterate whose weight is pending
    dx2 += IMPLICIT ? dd * dd / d.tw[j] : dd * dd;
  };
  spmv_rows<T, V, LANES>(d.n, d.t_ptr, d.t_col, d.t_val, y, d.t_thresh, d.t_long, d.t_nlong,
                         d.grid_p_short, epi);
  double v[1] = {(double)dx2}, out[1];
  block_sum<1>(v, out);
  if (threadIdx.x == 0) d.part_p[blockIdx.x] = out[0];
}

// A6: adaptive step-size rule, decided once per attempt by one thread.
__device__ __forceinline__ void decide_step(DevState* st, double dx2, double dy2, double dkd) {
  st->attempts += 1;
  const double k = (double)st->attempts;
  const double eta = st->eta, om = st->omega;
  if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(dkd)) {
    st->status = 4;  // PDLP_NUMERICAL
    return;
  }
  const double den = 2.0 * fabs(dkd);
  const double num = om * dx2 + dy2 / om;
  const double eta_bar = den > 0.0 ? num / den : INFINITY;
  bool accept = true;
  double eta_next = eta;
  if (st->adaptive) {
    eta_next = fmin((1.0 - pow(k + 1.0, -0.3)) * eta_bar, (1.0 + pow(k + 1.0, -0.6)) * eta);
    accept = !(eta > eta_bar);
  }
  const long long t = st->attempts - 1;
  if (t < st->tr_cap) {
    st->tr_eta[t] = eta;
    st->tr_eta_bar[t] = eta_bar;
    st->tr_accepted[t] = accept ? 1 : 0;
  }
  st->pending_w = 0.0;
  if (accept) {
    st->cur ^= 1;
    st->pending_w = eta;
    st->sum_w += eta;
    st->iters += 1;
    if (st->iters % st->period == 0 || st->iters >= st->iter_limit) st->check_due = 1;
  }
  st->eta = eta_next;
}

// ---------------------------------------------------------------- A5 + A6: dual
template <int LANES, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_dual(IterData<T, V> d) {
  DevState* st = d.st;
  if (st->status != 0 || st->check_due) return;
  const int cur = st->cur;
  const vec2_t<T>* __restrict__ xn = d.x[cur ^ 1];
  const T* __restrict__ y = d.y[cur];
  T* __restrict__ yn = d.y[cur ^ 1];
  const T sigma = (T)(st->eta * st->omega);
  const double pw64 = st->pending_w;
  const T pw = (T)pw64;
  T dy2 = 0, dkd = 0;
  // acc.a = (K x')_i, acc.b = (K dx)_i
  auto load = [&](int p) -> P2<T> {
    const T v = Ld<T, V>::get(d.a_val, p);
    const vec2_t<T> xv = xn[__ldg(d.a_col + p)];
    return P2<T>{v * xv.x, v * xv.y};
  };
  auto epi = [&](int i, P2<T> acc) {
    const T kxbar = acc.a + acc.b;  // K (2x' - x)
    const T yo = y[i];
    const T step = IMPLICIT ? sigma * d.sw[i] : sigma;
    T v = yo + step * (d.q[i] - kxbar);
    if (d.row_kind[i] != 1) v = maxv(v, (T)0);
    yn[i] = v;
    if (pw64 != 0.0) d.sum_y[i] += pw * yo;
    const T dd = v - yo;
    dy2 += IMPLICIT ? dd * dd / d.sw[i] : dd * dd;
    dkd += dd * acc.b;
  };
  if ((int)blockIdx.x < d.grid_d_short)
    rows_short<LANES, P2<T>>(d.m, d.a_ptr, d.a_thresh, d.grid_d_short, load, epi);
  else
    rows_long<P2<T>>(d.a_ptr, d.a_long, d.a_nlong, d.grid_d_short, load, epi);
  double v[2] = {(double)dy2, (double)dkd}, out[2];
  block_sum<2>(v, out);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    d.part_d[blockIdx.x] = out[0];
    d.part_d[d.grid_d + blockIdx.x] = out[1];
    __threadfence();
    last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sp[1], sd[2];
  {
    double a[1] = {0.0};
    for (int i = threadIdx.x; i < d.grid_p; i += kBlock) a[0] += __ldcg(d.part_p + i);
    block_sum<1>(a, sp);
    double b[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < d.grid_d; i += kBlock) {
      b[0] += __ldcg(d.part_d + i);
      b[1] += __ldcg(d.part_d + d.grid_d + i);
    }
    block_sum<2>(b, sd);
  }
  if (threadIdx.x == 0) {
    decide_step(st, sp[0], sd[0], sd[1]);
    st->counter = 0;
  }
}

}  // namespace pdlp
