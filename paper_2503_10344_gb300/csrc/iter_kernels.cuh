// Fused PDHG step kernels (rows A4-A7 of the hot path).
//
// One step attempt is two launches:
//   k_primal  -- CSR SpMV over A^T fused with the projected primal update
//                x' = proj_[l,u](x - tau (c - K^T y)) and the partial sums of
//                ||x' - x||^2 (scaled norm).
//   k_dual    -- CSR SpMV over A fused with the extrapolated dual update
//                y' = proj_Y(y + sigma (q - K(2x' - x))) and the partial sums
//                of ||y' - y||^2 and (y' - y)^T K (x' - x); its last block
//                reduces the partials in a fixed order and takes the adaptive
//                step-size decision (accept / retry) on the device.
// The primal iterate is stored as interleaved pairs (x'_j, x'_j - x_j): one
// vector gather per nonzero gives the dual kernel both K x' and K (x' - x),
// so K(2x' - x) = K x' + K dx and the step-size interaction term dy^T K dx are
// formed from K dx itself, not from the cancelling difference K x' - K x.
//
// Row traversal:
//   float32 iterates -- one aligned group of LANES lanes per row, rows
//     grid-strided (many warps in flight for the gathers); the group's first
//     lane runs the row's float32 epilogue.
//   float64 iterates -- a warp owns a tile of 32 consecutive rows, runs the
//     SpMV of the tile LANES lanes per row, stages the 32 row sums in shared
//     memory and then runs the 32 epilogues one per lane: on GB300 a float64
//     warp instruction costs the SM's FP64 pipe ~16 cycles however few lanes
//     are active, so the float64 epilogue must fill the warp.
// Rows longer than a threshold are handled by extra blocks at the end of the
// grid, one block per long row, so a skewed row cannot stall a group.
//
// The float32 kernels execute no float64 instruction: step sizes arrive
// prepared in float (DevState::tau_f ...), partial sums are reduced in float.
//
// Two storage forms (both are the same preconditioned iteration):
//   IMPLICIT = false: K~ = D_r K D_c is stored; vectors live in scaled space.
//   IMPLICIT = true : the unscaled K is stored (bfloat16 or a bare pattern) and
//                     the scaling is folded into per-element steps
//                     tau_j = tau D_c,j^2 (tw), sigma_i = sigma D_r,i^2 (sw);
//                     the scaled norms divide by tw / sw.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace pdlp {

__device__ __forceinline__ float clampv(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }
__device__ __forceinline__ double clampv(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }
__device__ __forceinline__ float maxv(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double maxv(double a, double b) { return fmax(a, b); }

// per-attempt scalars in the iterate type
template <typename T> struct StepT;
template <> struct StepT<float> {
  static __device__ __forceinline__ float tau(const DevState* s) { return s->tau_f; }
  static __device__ __forceinline__ float sigma(const DevState* s) { return s->sigma_f; }
  static __device__ __forceinline__ float pw(const DevState* s) { return s->pw_f; }
};
template <> struct StepT<double> {
  static __device__ __forceinline__ double tau(const DevState* s) { return s->tau_d; }
  static __device__ __forceinline__ double sigma(const DevState* s) { return s->sigma_d; }
  static __device__ __forceinline__ double pw(const DevState* s) { return s->pending_w; }
};

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
  T* part_p;                                           // [grid_p]
  T* part_d;                                           // [2][grid_d]
  int grid_p_short, grid_p, grid_d_short, grid_d;
  DevState* st;                                        // [count] (one per LP)
  Tables tp, td;                                       // batch tables over A^T / A (NULL: one LP)
};

// Rows of one LP (span), one aligned group of LANES lanes per row, rows
// grid-strided over the LP's short-row blocks; rows longer than `thresh` are
// skipped here (the long-row blocks own them).
template <int LANES, typename Acc, typename Load, typename Epi>
__device__ __forceinline__ void rows_short(const Span& sp, const int* __restrict__ ptr, int thresh,
                                           Load load, Epi epi) {
  const int lane = threadIdx.x & (LANES - 1);
  const long long G = (long long)sp.nshort * kBlock / LANES;
  const long long end = (long long)sp.row0 + sp.nrows;
  for (long long r = sp.row0 + ((long long)sp.bidx * kBlock + threadIdx.x) / LANES; r < end; r += G) {
    const int s = __ldg(ptr + r), e = __ldg(ptr + r + 1);
    if (e - s > thresh) continue;  // uniform within the group
    Acc acc{};
#pragma unroll 4  // independent index loads and gathers in flight per lane
    for (int p = s + lane; p < e; p += LANES) acc += load(p);
    acc = group_sum<LANES>(acc);
    if (lane == 0) epi((int)r, acc);
  }
}

// Tiles of 32 consecutive rows per warp: SpMV with LANES lanes per row in
// LANES passes, row sums staged in shared memory, then one epilogue per lane.
template <int LANES, typename Acc, typename Load, typename Epi>
__device__ __forceinline__ void rows_tiled(const Span& sp, const int* __restrict__ ptr, int thresh,
                                           Load load, Epi epi) {
  constexpr int GPW = 32 / LANES;  // rows per pass
  __shared__ Acc stage[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / LANES, gl = lane & (LANES - 1);
  const long long W = (long long)sp.nshort * kWarps;
  const long long end = (long long)sp.row0 + sp.nrows;
  for (long long t = (long long)sp.bidx * kWarps + warp; t * 32 < sp.nrows; t += W) {
    const long long r0 = sp.row0 + t * 32;
#pragma unroll 4
    for (int pass = 0; pass < LANES; ++pass) {
      const long long r = r0 + pass * GPW + g;
      Acc acc{};
      if (r < end) {
        const int s = __ldg(ptr + r), e = __ldg(ptr + r + 1);
        if (e - s <= thresh) {
#pragma unroll 4
          for (int p = s + gl; p < e; p += LANES) acc += load(p);
        }
      }
      acc = group_sum<LANES>(acc);
      if (gl == 0) stage[warp][pass * GPW + g] = acc;
    }
    __syncwarp();
    const long long r = r0 + lane;
    if (r < end) {
      const int s = __ldg(ptr + r), e = __ldg(ptr + r + 1);
      if (e - s <= thresh) epi((int)r, stage[warp][lane]);
    }
    __syncwarp();
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

// Long rows of the LP: one block per row of its list, its blocks [nshort, nblk).
template <typename Acc, typename Load, typename Epi>
__device__ __forceinline__ void rows_long(const Span& sp, const int* __restrict__ ptr, Load load,
                                          Epi epi) {
  for (int k = sp.bidx - sp.nshort; k < sp.nlist; k += sp.nblk - sp.nshort) {
    const int r = sp.list[k];
    const int s = ptr[r], e = ptr[r + 1];
    Acc acc{};
    for (int p = s + threadIdx.x; p < e; p += kBlock) acc += load(p);
    acc = block_allsum(acc);
    if (threadIdx.x == 0) epi(r, acc);
  }
}

// Short rows by groups (float) or warp tiles (double), long rows by blocks.
template <bool TILED, int LANES, typename Acc, typename Load, typename Epi>
__device__ __forceinline__ void rows_all(const Span& sp, const int* ptr, int thresh, Load load,
                                         Epi epi) {
  if (sp.bidx < sp.nshort) {
    if constexpr (TILED)
      rows_tiled<LANES, Acc>(sp, ptr, thresh, load, epi);
    else
      rows_short<LANES, Acc>(sp, ptr, thresh, load, epi);
  } else {
    rows_long<Acc>(sp, ptr, load, epi);
  }
}

// ---------------------------------------------------------------- A4: primal
template <int LANES, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_primal(IterData<T, V> d) {
  constexpr bool TILED = std::is_same<T, double>::value;
  const Span sp = make_span(d.tp, d.n, d.grid_p_short, d.t_long, d.t_nlong);
  DevState* st = d.st + sp.lp;
  if (st->status != 0 || st->check_due) return;
  const int cur = st->cur;
  const vec2_t<T>* __restrict__ x = cur ? d.x[1] : d.x[0];
  vec2_t<T>* __restrict__ xn = cur ? d.x[0] : d.x[1];
  const T* __restrict__ y = cur ? d.y[1] : d.y[0];
  const T tau = StepT<T>::tau(st);
  const T pw = StepT<T>::pw(st);
  T dx2 = 0;
  auto load = [&](int p) -> T { return Ld<T, V>::get(d.t_val, p) * __ldg(y + __ldg(d.t_col + p)); };
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
    if (pw != (T)0) d.sum_x[j] += pw * xo;  // A7: add the iterate whose weight is pending
    dx2 += IMPLICIT ? dd * dd / d.tw[j] : dd * dd;
  };
  rows_all<TILED, LANES, T>(sp, d.t_ptr, d.t_thresh, load, epi);
  const T s = block_sum1<T>(dx2);
  if (threadIdx.x == 0) d.part_p[blockIdx.x] = s;
}

// step-rule factors of attempt k (1-based)
__device__ __forceinline__ void step_factors(const DevState* st, long long k, double* fd, double* fi) {
  if (k <= st->fac_n) {
    *fd = st->fac_dec[k - 1];
    *fi = st->fac_inc[k - 1];
  } else {
    *fd = 1.0 - pow((double)k + 1.0, -0.3);
    *fi = 1.0 + pow((double)k + 1.0, -0.6);
  }
}

__device__ __forceinline__ void step_factors(const DevState* st, long long k, float* fd, float* fi) {
  if (k <= st->fac_n) {
    *fd = st->fac_dec_f[k - 1];
    *fi = st->fac_inc_f[k - 1];
  } else {
    *fd = 1.0f - powf((float)k + 1.0f, -0.3f);
    *fi = 1.0f + powf((float)k + 1.0f, -0.6f);
  }
}

// A6: adaptive step-size rule, decided once per attempt by one thread, in the
// iterate precision (float64 for the parity mode; float32 otherwise, with the
// float64 state mirrored for the restart logic and the report).
template <typename T>
__device__ __forceinline__ void decide_step(DevState* st, T dx2, T dy2, T dkd) {
  constexpr bool F64 = std::is_same<T, double>::value;
  st->attempts += 1;
  const long long k = st->attempts;
  if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(dkd)) {
    st->status = 4;  // PDLP_NUMERICAL
    return;
  }
  const T eta = F64 ? (T)st->eta : (T)st->eta_f;
  const T om = F64 ? (T)st->omega : (T)st->omega_f;
  const T iom = F64 ? (T)st->inv_omega : (T)st->inv_omega_f;
  const T den = (T)2 * fabs(dkd);
  // float64 (the parity mode) divides where the definition divides; float32
  // multiplies by the prepared reciprocal
  const T num = F64 ? om * dx2 + dy2 / om : om * dx2 + dy2 * iom;
  const T eta_bar = den > (T)0 ? num / den : (T)INFINITY;
  bool accept = true;
  T eta_next = eta;
  if (st->adaptive) {
    T fd, fi;
    step_factors(st, k, &fd, &fi);
    eta_next = fmin(fd * eta_bar, fi * eta);
    accept = !(eta > eta_bar);
  }
  const long long t = k - 1;
  if (t < st->tr_cap) {
    st->tr_eta[t] = (double)eta;
    st->tr_eta_bar[t] = (double)eta_bar;
    st->tr_accepted[t] = accept ? 1 : 0;
  }
  if (accept) {
    st->cur ^= 1;
    st->pending_w = (double)eta;
    st->pw_f = (float)eta;
    st->sum_w += (double)eta;
    st->iters += 1;
    if (st->iters % st->period == 0 || st->iters >= st->iter_limit) st->check_due = 1;
  } else {
    st->pending_w = 0.0;
    st->pw_f = 0.0f;
  }
  if (F64) {
    st->eta = (double)eta_next;
    st->tau_d = (double)(eta_next / om);
    st->sigma_d = (double)(eta_next * om);
  } else {
    st->eta_f = (float)eta_next;
    st->eta = (double)eta_next;
    st->tau_f = (float)(eta_next * iom);
    st->sigma_f = (float)(eta_next * om);
  }
}

// ---------------------------------------------------------------- A5 + A6: dual
template <int LANES, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_dual(IterData<T, V> d) {
  constexpr bool TILED = std::is_same<T, double>::value;
  const Span sp = make_span(d.td, d.m, d.grid_d_short, d.a_long, d.a_nlong);
  DevState* st = d.st + sp.lp;
  if (st->status != 0 || st->check_due) return;
  const int cur = st->cur;
  const vec2_t<T>* __restrict__ xn = cur ? d.x[0] : d.x[1];
  const T* __restrict__ y = cur ? d.y[1] : d.y[0];
  T* __restrict__ yn = cur ? d.y[0] : d.y[1];
  const T sigma = StepT<T>::sigma(st);
  const T pw = StepT<T>::pw(st);
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
    if (pw != (T)0) d.sum_y[i] += pw * yo;
    const T dd = v - yo;
    dy2 += IMPLICIT ? dd * dd / d.sw[i] : dd * dd;
    dkd += dd * acc.b;
  };
  rows_all<TILED, LANES, P2<T>>(sp, d.a_ptr, d.a_thresh, load, epi);
  const T s0 = block_sum1<T>(dy2);
  const T s1 = block_sum1<T>(dkd);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    d.part_d[blockIdx.x] = s0;
    d.part_d[d.grid_d + blockIdx.x] = s1;
    __threadfence();
    last = (atomicAdd(&st->counter, 1u) == (unsigned)sp.nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // this LP's partial slots: its primal blocks and its dual blocks
  int p0 = 0, pn = d.grid_p;
  if (d.tp.blk_lp != nullptr) {
    p0 = d.tp.blk0[sp.lp];
    pn = d.tp.nblk[sp.lp];
  }
  T a = 0, b0 = 0, b1 = 0;
  for (int i = threadIdx.x; i < pn; i += kBlock) a += __ldcg(d.part_p + p0 + i);
  for (int i = threadIdx.x; i < sp.nblk; i += kBlock) {
    b0 += __ldcg(d.part_d + sp.part0 + i);
    b1 += __ldcg(d.part_d + d.grid_d + sp.part0 + i);
  }
  block_sum3<T>(a, b0, b1);
  if (threadIdx.x == 0) {
    decide_step<T>(st, a, b0, b1);
    st->counter = 0;
  }
}

}  // namespace pdlp
