// One-block step kernel with the whole iteration problem in shared memory (rows A4-A7
// of the hot path for small LPs, pdlp_params.persistent = 2).
//
// The 200 x 400 MIP relaxations (1,600 nonzeros) leave a GPU-wide kernel nothing to
// spread: every step is a chain of dependent global loads (row pointer, column index,
// gathered entry) that a handful of warps cannot hide, and a launch per kernel costs as
// much as the work.  Here one block copies A and A^T (row pointers, column indices and
// values in the iterate type; none for a 0/1 pattern), the problem vectors and both
// iterate buffers into shared memory once per launch, then runs step attempts back to
// back until a KKT check falls due, the state stops the solve or `max_attempts` ran:
//   primal: x' = proj_[l,u](x - tau (c - K^T y)), one thread per column of A^T,
//           its entries summed in storage order; ||x' - x||^2;
//   dual:   y' = proj_Y(y + sigma (q - K(2x' - x))) from the (x', x' - x) pairs, one
//           thread per row of A; ||y' - y||^2 and (y' - y)^T K (x' - x);
//   decision (A6) by thread 0 on the block's copy of the state,
// with a block barrier between the phases.  The threads take the rows longest first (a
// stable order by length, built once per solve at setup), so the 32 rows of a warp have
// nearly equal lengths: a float64 warp instruction holds the SM's float64 pipe ~16
// cycles whatever its active lanes, and a warp's sum loop runs as long as its longest
// row.  At exit the iterate buffers and running sums go back to global memory (where
// the KKT block reads them) with the state.  The same iteration as the two-launch
// kernels; the partial sums are added in another order, so float64 iterates agree with
// theirs to rounding.
#pragma once

#include "internal.h"
#include "iter_kernels.cuh"

namespace pdlp {

template <typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_smem(IterData<T, V> d, SmemLayout L, int max_attempts) {
  constexpr bool VALS = !std::is_same<V, Pattern>::value;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ DevState ls;
  __shared__ int stop;
  __shared__ T red[3][kBlock];
  DevState* gst = d.st;
  if (threadIdx.x == 0) {
    ls = *gst;
    stop = (ls.status != 0 || ls.check_due) ? 1 : 0;
  }
  __syncthreads();
  if (stop) return;
  const int m = d.m, n = d.n, tid = threadIdx.x;
  int* tp = (int*)(sm + L.t_ptr);
  int* tc = (int*)(sm + L.t_col);
  T* tv = VALS ? (T*)(sm + L.t_val) : nullptr;
  int* ap = (int*)(sm + L.a_ptr);
  int* ac = (int*)(sm + L.a_col);
  T* av = VALS ? (T*)(sm + L.a_val) : nullptr;
  T* c = (T*)(sm + L.c);
  T* l = (T*)(sm + L.l);
  T* u = (T*)(sm + L.u);
  T* tw = IMPLICIT ? (T*)(sm + L.tw) : nullptr;
  T* q = (T*)(sm + L.q);
  T* sw = IMPLICIT ? (T*)(sm + L.sw) : nullptr;
  unsigned char* kind = sm + L.kind;
  vec2_t<T>* xs[2] = {(vec2_t<T>*)(sm + L.x0), (vec2_t<T>*)(sm + L.x1)};
  T* ys[2] = {(T*)(sm + L.y0), (T*)(sm + L.y1)};
  T* sx = (T*)(sm + L.sx);
  T* sy = (T*)(sm + L.sy);
  int* ot = (int*)(sm + L.ot);
  int* oa = (int*)(sm + L.oa);
  // ---- copy in (iterates with ordinary loads: the KKT block of the same graph wrote them)
  const int nnz = __ldg(d.t_ptr + n);
  for (int i = tid; i <= n; i += kBlock) tp[i] = __ldg(d.t_ptr + i);
  for (int i = tid; i <= m; i += kBlock) ap[i] = __ldg(d.a_ptr + i);
  // the order the threads take the columns and rows in (longest first, built at setup)
  for (int i = tid; i < n; i += kBlock) ot[i] = __ldg(d.ord_t + i);
  for (int i = tid; i < m; i += kBlock) oa[i] = __ldg(d.ord_a + i);
  for (int p = tid; p < nnz; p += kBlock) {
    tc[p] = __ldg(d.t_col + p);
    ac[p] = __ldg(d.a_col + p);
    if constexpr (VALS) {
      tv[p] = Ld<T, V>::get(d.t_val, p);
      av[p] = Ld<T, V>::get(d.a_val, p);
    }
  }
  for (int j = tid; j < n; j += kBlock) {
    c[j] = __ldg(d.c + j);
    l[j] = __ldg(d.l + j);
    u[j] = __ldg(d.u + j);
    if constexpr (IMPLICIT) tw[j] = __ldg(d.tw + j);
    xs[0][j] = d.x[0][j];
    xs[1][j] = d.x[1][j];
    sx[j] = d.sum_x[j];
  }
  for (int i = tid; i < m; i += kBlock) {
    q[i] = __ldg(d.q + i);
    if constexpr (IMPLICIT) sw[i] = __ldg(d.sw + i);
    kind[i] = __ldg(d.row_kind + i);
    ys[0][i] = d.y[0][i];
    ys[1][i] = d.y[1][i];
    sy[i] = d.sum_y[i];
  }
  __syncthreads();
  for (int att = 0; att < max_attempts; ++att) {
    const int cur = ls.cur;
    const T pw = StepT<T>::pw(&ls);
    const vec2_t<T>* x = xs[cur];
    vec2_t<T>* xn = xs[cur ^ 1];
    const T* y = ys[cur];
    T* yn = ys[cur ^ 1];
    // ---- A4: primal step, one thread per column
    const T tau = StepT<T>::tau(&ls);
    T dx2 = 0;
    for (int t = tid; t < n; t += kBlock) {
      const int j = ot[t];
      T aty = 0;
      for (int p = tp[j]; p < tp[j + 1]; ++p) aty += (VALS ? tv[p] : (T)1) * y[tc[p]];
      const T xo = x[j].x;
      const T step = IMPLICIT ? tau * tw[j] : tau;
      const T xv = clampv(xo - step * (c[j] - aty), l[j], u[j]);
      const T dd = xv - xo;
      vec2_t<T> o;
      o.x = xv;
      o.y = dd;
      xn[j] = o;
      if (pw != (T)0) sx[j] += pw * xo;  // A7: add the iterate whose weight is pending
      dx2 += IMPLICIT ? dd * dd / tw[j] : dd * dd;
    }
    __syncthreads();  // xn complete before the dual phase gathers it
    // ---- A5: dual step, one thread per row
    const T sigma = StepT<T>::sigma(&ls);
    T dy2 = 0, dkd = 0;
    for (int t = tid; t < m; t += kBlock) {
      const int i = oa[t];
      T kx = 0, kd = 0;  // (K x')_i, (K dx)_i
      for (int p = ap[i]; p < ap[i + 1]; ++p) {
        const T v = VALS ? av[p] : (T)1;
        const vec2_t<T> xv = xn[ac[p]];
        kx += v * xv.x;
        kd += v * xv.y;
      }
      const T yo = y[i];
      const T step = IMPLICIT ? sigma * sw[i] : sigma;
      T yv = yo + step * (q[i] - (kx + kd));
      if (kind[i] != 1) yv = maxv(yv, (T)0);
      yn[i] = yv;
      if (pw != (T)0) sy[i] += pw * yo;
      const T dd = yv - yo;
      dy2 += IMPLICIT ? dd * dd / sw[i] : dd * dd;
      dkd += dd * kd;
    }
    // the three sums by one warp: every thread's values through shared memory, eight
    // additions per lane, then five shuffle levels (a float64 warp instruction holds the
    // pipe as long with one active lane as with 32, so one warp reducing costs an eighth
    // of eight warps shuffling)
    red[0][tid] = dx2;
    red[1][tid] = dy2;
    red[2][tid] = dkd;
    __syncthreads();
    if (tid < 32) {
      T a = 0, b0 = 0, b1 = 0;
#pragma unroll
      for (int i = tid; i < kBlock; i += 32) {
        a += red[0][i];
        b0 += red[1][i];
        b1 += red[2][i];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b0 += __shfl_xor_sync(0xffffffffu, b0, o);
        b1 += __shfl_xor_sync(0xffffffffu, b1, o);
      }
      // ---- A6: the decision
      if (tid == 0) {
        T fd, fi;
        step_factors(&ls, ls.attempts + 1, &fd, &fi);
        decide_step<T>(&ls, a, b0, b1, fd, fi);
      }
    }
    __syncthreads();
    if (ls.status != 0 || ls.check_due) break;
  }
  // ---- copy out
  for (int j = tid; j < n; j += kBlock) {
    d.x[0][j] = xs[0][j];
    d.x[1][j] = xs[1][j];
    d.sum_x[j] = sx[j];
  }
  for (int i = tid; i < m; i += kBlock) {
    d.y[0][i] = ys[0][i];
    d.y[1][i] = ys[1][i];
    d.sum_y[i] = sy[i];
  }
  if (tid == 0) store_step_state(gst, ls);
}

}  // namespace pdlp
