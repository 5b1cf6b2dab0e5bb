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
  unsigned* cnt;                                       // [count][kCountGroups][8] group counters
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

// Two rows per group and pass, rows g and g + G of the grid's G groups, their
// index loads and gathers interleaved in one loop (twice the loads in flight of
// one row at a time), and each row's epilogue operands fetched by the epilogue
// lane before the SpMV (they depend on the row index only), so the epilogue
// does not add a round trip after the gathers.  `pref(r)` returns the operands,
// `epi(r, acc, pre)` finishes the row.  Rows longer than `thresh` are skipped.
template <int LANES, typename Acc, typename Pre, typename Load, typename PreF, typename Epi>
__device__ __forceinline__ void rows_short2(const Span& sp, const int* __restrict__ ptr, int thresh,
                                            Load load, PreF pref, Epi epi) {
  const int lane = threadIdx.x & (LANES - 1);
  const long long G = (long long)sp.nshort * kBlock / LANES;
  const long long end = (long long)sp.row0 + sp.nrows;
  for (long long r0 = sp.row0 + ((long long)sp.bidx * kBlock + threadIdx.x) / LANES; r0 < end;
       r0 += 2 * G) {
    const long long r1 = r0 + G;
    const bool has1 = r1 < end;
    int s0 = __ldg(ptr + r0), e0 = __ldg(ptr + r0 + 1);
    int s1 = 0, e1 = 0;
    if (has1) {
      s1 = __ldg(ptr + r1);
      e1 = __ldg(ptr + r1 + 1);
    }
    const bool ok0 = e0 - s0 <= thresh;  // uniform within the group
    const bool ok1 = has1 && e1 - s1 <= thresh;
    const int n0 = ok0 ? e0 - s0 : 0, n1 = ok1 ? e1 - s1 : 0;
    Pre p0{}, p1{};
    if (lane == 0) {
      if (ok0) p0 = pref((int)r0);
      if (ok1) p1 = pref((int)r1);
    }
    Acc a0{}, a1{};
    const int nmax = n0 > n1 ? n0 : n1;
#pragma unroll 2
    for (int k = lane; k < nmax; k += LANES) {
      if (k < n0) a0 += load(s0 + k);
      if (k < n1) a1 += load(s1 + k);
    }
    a0 = group_sum<LANES>(a0);
    a1 = group_sum<LANES>(a1);
    if (lane == 0) {
      if (ok0) epi((int)r0, a0, p0);
      if (ok1) epi((int)r1, a1, p1);
    }
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
// resident blocks per SM the float32 step kernels are compiled for (register
// budget 42): the float32 solve of the 50k x 200k covering LP needs 782 blocks
// for one pass, six per SM keep them all resident; the float64 kernels keep
// their registers (a tighter budget spills)
template <typename T> struct StepOcc { static constexpr int value = 6; };
template <> struct StepOcc<double> { static constexpr int value = 1; };

// group counters of the dual kernel's last-block detection (per LP)
constexpr int kCountGroups = 32;

template <typename T>
struct PreP {  // epilogue operands of a primal row
  T xo, c, l, u, tw, sx;
};
template <typename T>
struct PreD {  // epilogue operands of a dual row
  T yo, q, sw, sy;
  int kind;
};

template <int LANES, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock, StepOcc<T>::value) k_primal(IterData<T, V> d) {
  pdl_enter();
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
  auto pref = [&](int j) -> PreP<T> {
    PreP<T> o;
    o.xo = x[j].x;
    o.c = d.c[j];
    o.l = d.l[j];
    o.u = d.u[j];
    o.tw = IMPLICIT ? d.tw[j] : (T)1;
    o.sx = pw != (T)0 ? d.sum_x[j] : (T)0;
    return o;
  };
  auto fin = [&](int j, T aty, const PreP<T>& o) {
    const T g = o.c - aty;
    const T step = IMPLICIT ? tau * o.tw : tau;
    const T xv = clampv(o.xo - step * g, o.l, o.u);
    const T dd = xv - o.xo;
    vec2_t<T> v;
    v.x = xv;
    v.y = dd;
    xn[j] = v;
    if (pw != (T)0) d.sum_x[j] = o.sx + pw * o.xo;  // A7: add the iterate whose weight is pending
    dx2 += IMPLICIT ? dd * dd / o.tw : dd * dd;
  };
  auto epi = [&](int j, T aty) { fin(j, aty, pref(j)); };
  if constexpr (TILED) {
    rows_all<true, LANES, T>(sp, d.t_ptr, d.t_thresh, load, epi);
  } else {
    if (sp.bidx < sp.nshort)
      rows_short2<LANES, T, PreP<T>>(sp, d.t_ptr, d.t_thresh, load, pref, fin);
    else
      rows_long<T>(sp, d.t_ptr, load, epi);
  }
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
// iterate precision; fd, fi are the step-rule factors of this attempt
// (k = attempts + 1), fetched by the caller ahead of time.  In the
// iterate precision (float64 for the parity mode; float32 otherwise, with the
// float64 state mirrored for the restart logic and the report).
template <typename T>
__device__ __forceinline__ void decide_step(DevState* st, T dx2, T dy2, T dkd, T fd, T fi) {
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

// fields of the state a step decision changes (the barrier words are not copied)
__device__ __forceinline__ void store_step_state(DevState* g, const DevState& l) {
  g->status = l.status;
  g->check_due = l.check_due;
  g->iters = l.iters;
  g->attempts = l.attempts;
  g->eta = l.eta;
  g->sum_w = l.sum_w;
  g->pending_w = l.pending_w;
  g->cur = l.cur;
  g->tau_d = l.tau_d;
  g->sigma_d = l.sigma_d;
  g->tau_f = l.tau_f;
  g->sigma_f = l.sigma_f;
  g->pw_f = l.pw_f;
  g->eta_f = l.eta_f;
}

// ---------------------------------------------------------------- A5 + A6: dual
template <int LANES, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock, StepOcc<T>::value) k_dual(IterData<T, V> d) {
  pdl_enter();
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
  // the state and this attempt's step-rule factors, taken at entry: if this
  // block turns out to be the LP's last, its decision needs no further load
  __shared__ DevState ls;
  __shared__ T fac[2];
  if (threadIdx.x == 0) {
    ls = *st;
    step_factors(&ls, ls.attempts + 1, &fac[0], &fac[1]);
  }
  T dy2 = 0, dkd = 0;
  // acc.a = (K x')_i, acc.b = (K dx)_i
  auto load = [&](int p) -> P2<T> {
    const T v = Ld<T, V>::get(d.a_val, p);
    const vec2_t<T> xv = xn[__ldg(d.a_col + p)];
    return P2<T>{v * xv.x, v * xv.y};
  };
  auto pref = [&](int i) -> PreD<T> {
    PreD<T> o;
    o.yo = y[i];
    o.q = d.q[i];
    o.sw = IMPLICIT ? d.sw[i] : (T)1;
    o.sy = pw != (T)0 ? d.sum_y[i] : (T)0;
    o.kind = d.row_kind[i];
    return o;
  };
  auto fin = [&](int i, P2<T> acc, const PreD<T>& o) {
    const T kxbar = acc.a + acc.b;  // K (2x' - x)
    const T step = IMPLICIT ? sigma * o.sw : sigma;
    T v = o.yo + step * (o.q - kxbar);
    if (o.kind != 1) v = maxv(v, (T)0);
    yn[i] = v;
    if (pw != (T)0) d.sum_y[i] = o.sy + pw * o.yo;
    const T dd = v - o.yo;
    dy2 += IMPLICIT ? dd * dd / o.sw : dd * dd;
    dkd += dd * acc.b;
  };
  auto epi = [&](int i, P2<T> acc) { fin(i, acc, pref(i)); };
  if constexpr (TILED) {
    rows_all<true, LANES, P2<T>>(sp, d.a_ptr, d.a_thresh, load, epi);
  } else {
    if (sp.bidx < sp.nshort)
      rows_short2<LANES, P2<T>, PreD<T>>(sp, d.a_ptr, d.a_thresh, load, pref, fin);
    else
      rows_long<P2<T>>(sp, d.a_ptr, load, epi);
  }
  const T s0 = block_sum1<T>(dy2);
  const T s1 = block_sum1<T>(dkd);
  // Last-block detection in two levels, so that the blocks finishing together do
  // not queue on one address: block b of the LP counts on group counter
  // b % ng (ng = min(32, blocks), each on its own 32-byte sector); the last of
  // a group resets it and counts on the LP's counter; the last of those decides.
  __shared__ bool last;
  if (threadIdx.x == 0) {
    d.part_d[blockIdx.x] = s0;
    d.part_d[d.grid_d + blockIdx.x] = s1;
    __threadfence();
    const int ng = sp.nblk < kCountGroups ? sp.nblk : kCountGroups;
    const int g = sp.bidx % ng;
    const unsigned gsize = (unsigned)((sp.nblk - g + ng - 1) / ng);
    unsigned* gc = d.cnt + ((size_t)sp.lp * kCountGroups + g) * 8;
    bool top = false;
    if (atomicAdd(gc, 1u) == gsize - 1) {
      *gc = 0u;  // every member of the group has counted this attempt
      __threadfence();
      top = atomicAdd(&st->counter, 1u) == (unsigned)ng - 1;
    }
    last = top;
  }
  __syncthreads();
  if (!last) return;
  if (st->dry) {  // shape tuning: the iterate and the state stay as they were
    if (threadIdx.x == 0) st->counter = 0;
    return;
  }
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
    decide_step<T>(&ls, a, b0, b1, fac[0], fac[1]);
    store_step_state(st, ls);
    st->counter = 0;
  }
}

// ---------------------------------------------------------------- persistent attempts
// One cooperative launch (every block resident) runs step attempts until a KKT
// check falls due, the state stops the solve, or `max_attempts` have run.  An
// attempt is the primal phase (A4), a grid barrier, the dual phase (A5), a grid
// barrier, and the step decision (A6) -- taken by EVERY block from the same
// partial sums in the same order, so all blocks hold bit-identical copies of
// the step state in shared memory and no third barrier is needed; block 0
// records the decision trace and writes the state back at exit.  Rows keep
// their owner thread across attempts, so a row's own iterate entries are read
// back by the thread that wrote them; entries gathered from other blocks' rows
// (y in the primal phase, the (x', dx) pairs in the dual phase) and the
// partial sums are read through L2 (ld.global.cg), never through the
// non-coherent L1 path.  Partial sums alternate between two buffers by attempt
// parity, so a block still reducing attempt k never sees attempt k + 1's
// values.  Every barrier wait is bounded: a block that gives up flags the
// state (kStatusWaitFailed) and returns, and so do the others.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

constexpr long long kSpinLimit = 1LL << 23;  // polls of one barrier wait (seconds)

__device__ __forceinline__ bool grid_barrier(DevState* st) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(&st->bar_gen);
    __threadfence();
    int good = 1;
    if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long polls = 0;
      while (ld_acquire_u32(&st->bar_gen) == gen) {
        if (++polls > kSpinLimit || *(volatile int*)&st->bar_err) {
          good = 0;
          break;
        }
      }
    }
    if (!good) {
      atomicExch(&st->bar_err, 1);
      atomicExch(&st->status, kStatusWaitFailed);
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <int LA, int LT, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_persist(IterData<T, V> d, int max_attempts) {
  constexpr bool TILED = std::is_same<T, double>::value;
  DevState* gst = d.st;
  __shared__ DevState ls;
  __shared__ int stop;
  if (threadIdx.x == 0) {
    ls = *gst;
    if (blockIdx.x != 0) ls.tr_cap = 0;  // one block writes the trace
    stop = (ls.status != 0 || ls.check_due) ? 1 : 0;
  }
  __syncthreads();
  if (stop) return;
  const int G = gridDim.x;
  const int b = blockIdx.x;
  T* pp = d.part_p;  // [2][G]
  T* pd = d.part_d;  // [2][2][G]
  const Span sp_p{0, 0, d.n, b, G, G, 0, d.t_long, d.t_nlong};
  const Span sp_pl{0, 0, d.n, b, 0, G, 0, d.t_long, d.t_nlong};
  const Span sp_d{0, 0, d.m, b, G, G, 0, d.a_long, d.a_nlong};
  const Span sp_dl{0, 0, d.m, b, 0, G, 0, d.a_long, d.a_nlong};
  for (int att = 0; att < max_attempts; ++att) {
    const int par = (int)(ls.attempts & 1);
    const int cur = ls.cur;
    const T pw = StepT<T>::pw(&ls);
    // ---- A4: primal step over the rows of A^T
    {
      const vec2_t<T>* x = cur ? d.x[1] : d.x[0];
      vec2_t<T>* xn = cur ? d.x[0] : d.x[1];
      const T* y = cur ? d.y[1] : d.y[0];
      const T tau = StepT<T>::tau(&ls);
      T dx2 = 0;
      auto load = [&](int p) -> T {
        return Ld<T, V>::get(d.t_val, p) * __ldcg(y + __ldg(d.t_col + p));
      };
      auto epi = [&](int j, T aty) {
        const T xo = __ldcg(x + j).x;
        const T g = __ldg(d.c + j) - aty;
        const T step = IMPLICIT ? tau * __ldg(d.tw + j) : tau;
        const T xv = clampv(xo - step * g, __ldg(d.l + j), __ldg(d.u + j));
        const T dd = xv - xo;
        vec2_t<T> o;
        o.x = xv;
        o.y = dd;
        xn[j] = o;
        if (pw != (T)0) d.sum_x[j] = __ldcg(d.sum_x + j) + pw * xo;
        dx2 += IMPLICIT ? dd * dd / __ldg(d.tw + j) : dd * dd;
      };
      if constexpr (TILED)
        rows_tiled<LT, T>(sp_p, d.t_ptr, d.t_thresh, load, epi);
      else
        rows_short<LT, T>(sp_p, d.t_ptr, d.t_thresh, load, epi);
      rows_long<T>(sp_pl, d.t_ptr, load, epi);
      const T s = block_sum1<T>(dx2);
      if (threadIdx.x == 0) pp[par * G + b] = s;
    }
    if (!grid_barrier(gst)) return;
    // ---- A5: dual step over the rows of A
    {
      const vec2_t<T>* xn = cur ? d.x[0] : d.x[1];
      const T* y = cur ? d.y[1] : d.y[0];
      T* yn = cur ? d.y[0] : d.y[1];
      const T sigma = StepT<T>::sigma(&ls);
      T dy2 = 0, dkd = 0;
      auto load = [&](int p) -> P2<T> {
        const T v = Ld<T, V>::get(d.a_val, p);
        const vec2_t<T> xv = __ldcg(xn + __ldg(d.a_col + p));
        return P2<T>{v * xv.x, v * xv.y};
      };
      auto epi = [&](int i, P2<T> acc) {
        const T kxbar = acc.a + acc.b;
        const T yo = __ldcg(y + i);
        const T step = IMPLICIT ? sigma * __ldg(d.sw + i) : sigma;
        T v = yo + step * (__ldg(d.q + i) - kxbar);
        if (__ldg(d.row_kind + i) != 1) v = maxv(v, (T)0);
        yn[i] = v;
        if (pw != (T)0) d.sum_y[i] = __ldcg(d.sum_y + i) + pw * yo;
        const T dd = v - yo;
        dy2 += IMPLICIT ? dd * dd / __ldg(d.sw + i) : dd * dd;
        dkd += dd * acc.b;
      };
      if constexpr (TILED)
        rows_tiled<LA, P2<T>>(sp_d, d.a_ptr, d.a_thresh, load, epi);
      else
        rows_short<LA, P2<T>>(sp_d, d.a_ptr, d.a_thresh, load, epi);
      rows_long<P2<T>>(sp_dl, d.a_ptr, load, epi);
      const T s0 = block_sum1<T>(dy2);
      const T s1 = block_sum1<T>(dkd);
      if (threadIdx.x == 0) {
        pd[(2 * par) * G + b] = s0;
        pd[(2 * par + 1) * G + b] = s1;
      }
    }
    if (!grid_barrier(gst)) return;
    // ---- A6: the same decision in every block
    {
      T a = 0, b0 = 0, b1 = 0;
      for (int i = threadIdx.x; i < G; i += kBlock) {
        a += __ldcg(pp + par * G + i);
        b0 += __ldcg(pd + (2 * par) * G + i);
        b1 += __ldcg(pd + (2 * par + 1) * G + i);
      }
      block_sum3<T>(a, b0, b1);
      if (threadIdx.x == 0) {
        T fd, fi;
        step_factors(&ls, ls.attempts + 1, &fd, &fi);
        decide_step<T>(&ls, a, b0, b1, fd, fi);
      }
      __syncthreads();
    }
    if (ls.status != 0 || ls.check_due) break;
  }
  if (b == 0 && threadIdx.x == 0) store_step_state(gst, ls);
}

}  // namespace pdlp
