// Fused PDHG step kernels (rows A4-A7 of the hot path).
//
// One step attempt is two launches:
//   k_primal  -- CSR SpMV over A^T fused with the projected primal update
//                x' = proj_[l,u](x - tau (c - K^T y)) and the partial sums of
//                ||x' - x||^2 (scaled norm).
//   k_dual    -- CSR SpMV over A fused with the extrapolated dual update
//                y' = proj_Y(y + sigma (q - K(2x' - x))) and the partial sums
//                of ||y' - y||^2 and (y' - y)^T K (x' - x);
//   k_decide  -- one block per LP: the partial sums in a fixed order and the
//                adaptive step-size decision (accept / retry) on the device.
// All three are launched with programmatic dependent launch (see common.cuh).
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
  static __device__ __forceinline__ float ha(const DevState* s) { return s->ha_f; }
  static __device__ __forceinline__ float hb(const DevState* s) { return s->hb_f; }
  static __device__ __forceinline__ float hc(const DevState* s) { return s->hc_f; }
};
template <> struct StepT<double> {
  static __device__ __forceinline__ double tau(const DevState* s) { return s->tau_d; }
  static __device__ __forceinline__ double sigma(const DevState* s) { return s->sigma_d; }
  static __device__ __forceinline__ double pw(const DevState* s) { return s->pending_w; }
  static __device__ __forceinline__ double ha(const DevState* s) { return s->ha_d; }
  static __device__ __forceinline__ double hb(const DevState* s) { return s->hb_d; }
  static __device__ __forceinline__ double hc(const DevState* s) { return s->hc_d; }
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
  int count;                                           // LPs (1 for a single LP)
  unsigned long long cond;                             // while-loop handle of the graph (0: none)
  int loop_cap;                                        // attempts per graph launch at most
  Tables tp, td;                                       // batch tables over A^T / A (NULL: one LP)
  int tile;                                            // tile kernels (float32 only): form
  TileSet tt, ta;                                      // their items over A^T and A
  int grid_tt, grid_ta, work_tt, work_ta, tslot;
  const int *ord_t, *ord_a;                            // one-block kernel: rows longest first
  // Halpern variant (H kernels): the iterate z = (hx, hy) the step starts from, updated in
  // place by the row's owner, and the anchor (hax, hay)
  T* hx; T* hy; const T* hax; const T* hay;
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

// Two rows per group and pass, rows g and g + G of the grid's G groups, their loads
// interleaved (twice the loads in flight of one row at a time), software-pipelined
// across passes: while a pass gathers and finishes its row pair, each lane's first
// kPre column indices and values of the next pair's rows (from row pointers loaded
// one pass earlier) and the row pointers of the pair after it are already in
// flight, so a pass waits on its gathers alone instead of on the row pointer ->
// column index -> gather chain; entries beyond kPre per lane follow in a dependent
// loop.  The first pair's pointers, indices and values and the second pair's
// pointers are loaded BEFORE `enter()` waits for the preceding kernel (they do not
// depend on the iterate).  The epilogue operands (`pref_c` constant, `pref_v`
// iterate) are issued alongside the gathers.  `enter()` returns false when the state
// says the kernel has nothing to do (uniform over the block).  `val(p)` is the
// stored value at position p, `term(v, j)` the row-sum term of value v and gathered
// entry j, `fin(r, acc, pc, pv)` finishes a row.  Rows longer than `thresh` are
// skipped (long-row blocks own them).  (A prefetch depth of 4 measured slower:
// register spills at the 64 registers of four blocks per SM.)  With one lane per row
// every thread finishes its own rows (no idle lanes in the epilogue, consecutive rows
// on consecutive lanes) and prefetches kPre1 entries of each.
constexpr int kPre = 2;
constexpr int kPre1 = 3;
// one lane per row in the dual kernel: the entries past the first kPre1 are loaded kChunk1
// at a time before their gathers (the energy model's 175,200 balance rows of 13-21 entries
// come first in row order and make the first pass long: dual half-step 42.8 -> 41.1 us;
// in the primal kernel the chunk's registers delayed the next pass's prefetch instead)
constexpr int kChunk1 = 4;
template <int LANES> struct PreDepth { static constexpr int value = LANES == 1 ? kPre1 : kPre; };

template <int LANES, typename Acc, typename PC, typename PV, bool CHUNK_TAIL = false, typename Val,
          typename Term, typename PrefC, typename PrefV, typename Fin, typename Enter>
__device__ __forceinline__ bool rows_short3(const Span& sp, const int* __restrict__ ptr,
                                            const int* __restrict__ col, int thresh, Val val,
                                            Term term, PrefC pref_c, PrefV pref_v, Fin fin,
                                            Enter enter) {
  using VT = decltype(val(0));
  constexpr int KP = PreDepth<LANES>::value;
  const int lane = threadIdx.x & (LANES - 1);
  const long long G = (long long)sp.nshort * kBlock / LANES;
  const long long end = (long long)sp.row0 + sp.nrows;
  long long r0 = sp.row0 + ((long long)sp.bidx * kBlock + threadIdx.x) / LANES;
  struct Rows {  // a pair's starts and lengths (-1: a long row or no row)
    int s0, n0, s1, n1;
  };
  struct Heads {  // each lane's first KP column indices and values of the pair's rows
    int c0[KP], c1[KP];
    VT v0[KP], v1[KP];
  };
  auto load_rows = [&](long long ra) -> Rows {
    Rows p{0, -1, 0, -1};
    if (ra < end) {
      const int s = __ldg(ptr + ra), e = __ldg(ptr + ra + 1);
      p.s0 = s;
      p.n0 = e - s <= thresh ? e - s : -1;
    }
    if (ra + G < end) {
      const int s = __ldg(ptr + ra + G), e = __ldg(ptr + ra + G + 1);
      p.s1 = s;
      p.n1 = e - s <= thresh ? e - s : -1;
    }
    return p;
  };
  auto load_heads = [&](const Rows& p) -> Heads {
    Heads h;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int q = lane + k * LANES;
      h.c0[k] = q < p.n0 ? __ldg(col + p.s0 + q) : 0;
      h.v0[k] = q < p.n0 ? val(p.s0 + q) : VT(0);
      h.c1[k] = q < p.n1 ? __ldg(col + p.s1 + q) : 0;
      h.v1[k] = q < p.n1 ? val(p.s1 + q) : VT(0);
    }
    return h;
  };
  Rows rw = load_rows(r0);
  Heads hd = load_heads(rw);
  Rows rn = load_rows(r0 + 2 * G);
  if (!enter()) return false;
  for (; r0 < end; r0 += 2 * G) {
    const long long r1 = r0 + G;
    // the next pair's heads and the pointers of the pair after it: independent of
    // this pair's gathers, issued first
    const Heads hn = load_heads(rn);
    const Rows rnn = load_rows(r0 + 4 * G);
    PC pc0{}, pc1{};
    PV pv0{}, pv1{};
    if (lane == 0) {
      if (rw.n0 >= 0) {
        pc0 = pref_c((int)r0);
        pv0 = pref_v((int)r0);
      }
      if (rw.n1 >= 0) {
        pc1 = pref_c((int)r1);
        pv1 = pref_v((int)r1);
      }
    }
    Acc a0{}, a1{};
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int q = lane + k * LANES;
      if (q < rw.n0) a0 += term(hd.v0[k], hd.c0[k]);
      if (q < rw.n1) a1 += term(hd.v1[k], hd.c1[k]);
    }
    const int nmax = rw.n0 > rw.n1 ? rw.n0 : rw.n1;
    if constexpr (LANES == 1 && CHUNK_TAIL) {
      // a thread walks the rest of its two rows alone: kChunk1 indices and values of
      // each issued together, then their gathers (the same order of the sums; with more
      // lanes per row the chunks measured slower: covering LP dual 11.7 -> 12.0 us, batch
      // dual 595 -> 617 us)
      for (int q0 = KP; q0 < nmax; q0 += kChunk1) {
        int c0[kChunk1], c1[kChunk1];
        VT v0[kChunk1], v1[kChunk1];
#pragma unroll
        for (int k = 0; k < kChunk1; ++k) {
          const int q = q0 + k;
          c0[k] = q < rw.n0 ? __ldg(col + rw.s0 + q) : -1;
          v0[k] = q < rw.n0 ? val(rw.s0 + q) : VT(0);
          c1[k] = q < rw.n1 ? __ldg(col + rw.s1 + q) : -1;
          v1[k] = q < rw.n1 ? val(rw.s1 + q) : VT(0);
        }
#pragma unroll
        for (int k = 0; k < kChunk1; ++k) {
          if (c0[k] >= 0) a0 += term(v0[k], c0[k]);
          if (c1[k] >= 0) a1 += term(v1[k], c1[k]);
        }
      }
    } else {
#pragma unroll 2
      for (int q = lane + KP * LANES; q < nmax; q += LANES) {
        if (q < rw.n0) a0 += term(val(rw.s0 + q), __ldg(col + rw.s0 + q));
        if (q < rw.n1) a1 += term(val(rw.s1 + q), __ldg(col + rw.s1 + q));
      }
    }
    a0 = group_sum<LANES>(a0);
    a1 = group_sum<LANES>(a1);
    if (lane == 0) {
      if (rw.n0 >= 0) fin((int)r0, a0, pc0, pv0);
      if (rw.n1 >= 0) fin((int)r1, a1, pc1, pv1);
    }
    rw = rn;
    hd = hn;
    rn = rnn;
  }
  return true;
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
// resident blocks per SM the float32 step kernels are compiled for (kStepBlocksPerSmF32,
// a 64-register budget: the pipelined traversal holds two passes of row pointers and one
// of column indices and values per lane); the float64 kernels keep their registers (a
// tighter budget spills)
template <typename T> struct StepOcc { static constexpr int value = kStepBlocksPerSmF32; };
template <> struct StepOcc<double> { static constexpr int value = 1; };

// epilogue operands of a row: constant ones (read before the dependent-launch
// wait) and iterate ones (after it)
template <typename T>
struct PreCP {  // primal row j: c, l, u, step weight
  T c, l, u, tw;
};
template <typename T>
struct PreVP {  // primal row j: x_j, running sum
  T xo, sx;
};
template <typename T>
struct PreCD {  // dual row i: q, step weight, row kind
  T q, sw;
  int kind;
};
template <typename T>
struct PreVD {  // dual row i: y_i, running sum
  T yo, sy;
};

// Iterate vectors written by the preceding kernels are read with ordinary
// (weak, L1-cacheable) loads after the dependent-launch wait, whose guarantee
// covers them; never through the non-coherent read-only path (__ldg), which
// assumes data that no grid in flight writes.
//
// H (the Halpern variant, pdlp_params.halpern): the step starts from the Halpern iterate
// (hx, hy) instead of the current buffers, writes T(z) as usual (the (x', dx) pairs and
// y' in the next buffers: the candidate the checks evaluate), and each row's owner
// replaces its entry of the Halpern iterate by ha T(z) + hb z + hc z_a; no averages.
template <int LANES, typename T, typename V, bool IMPLICIT, bool H = false>
__global__ void __launch_bounds__(kBlock, StepOcc<T>::value) k_primal(IterData<T, V> d) {
  constexpr bool TILED = std::is_same<T, double>::value;
  const Span sp = make_span(d.tp, d.n, d.grid_p_short, d.t_long, d.t_nlong);
  DevState* st = d.st + sp.lp;
  const vec2_t<T>* x = nullptr;
  vec2_t<T>* xn = nullptr;
  const T* y = nullptr;
  T tau = 0, pw = 0, ha = 0, hb = 0, hc = 0;
  auto enter = [&]() -> bool {
    pdl_enter();
    if (st->status != 0 || st->check_due) return false;
    const int cur = st->cur;
    x = cur ? d.x[1] : d.x[0];
    xn = cur ? d.x[0] : d.x[1];
    y = H ? d.hy : cur ? d.y[1] : d.y[0];
    tau = StepT<T>::tau(st);
    if constexpr (H) {
      ha = StepT<T>::ha(st);
      hb = StepT<T>::hb(st);
      hc = StepT<T>::hc(st);
    } else {
      pw = StepT<T>::pw(st);
    }
    return true;
  };
  T dx2 = 0;
  auto val = [&](int p) -> T { return Ld<T, V>::get(d.t_val, p); };
  auto term = [&](T v, int i) -> T { return v * y[i]; };
  auto load = [&](int p) -> T { return term(val(p), __ldg(d.t_col + p)); };
  auto pref_c = [&](int j) -> PreCP<T> {
    return PreCP<T>{__ldg(d.c + j), __ldg(d.l + j), __ldg(d.u + j), IMPLICIT ? __ldg(d.tw + j) : (T)1};
  };
  auto pref_v = [&](int j) -> PreVP<T> {
    if constexpr (H) return PreVP<T>{d.hx[j], d.hax[j]};  // the iterate and its anchor
    return PreVP<T>{x[j].x, pw != (T)0 ? d.sum_x[j] : (T)0};
  };
  auto fin = [&](int j, T aty, const PreCP<T>& c, const PreVP<T>& v) {
    const T g = c.c - aty;
    const T step = IMPLICIT ? tau * c.tw : tau;
    const T xv = clampv(v.xo - step * g, c.l, c.u);
    const T dd = xv - v.xo;
    vec2_t<T> o;
    o.x = xv;
    o.y = dd;
    xn[j] = o;
    if constexpr (H)
      d.hx[j] = ha * xv + hb * v.xo + hc * v.sx;  // the reflected Halpern mix
    else if (pw != (T)0)
      d.sum_x[j] = v.sx + pw * v.xo;  // A7: add the iterate whose weight is pending
    dx2 += IMPLICIT ? dd * dd / c.tw : dd * dd;
  };
  auto epi = [&](int j, T aty) { fin(j, aty, pref_c(j), pref_v(j)); };
  if constexpr (TILED) {
    if (!enter()) return;
    rows_all<true, LANES, T>(sp, d.t_ptr, d.t_thresh, load, epi);
  } else if (sp.bidx < sp.nshort) {
    if (!rows_short3<LANES, T, PreCP<T>, PreVP<T>>(sp, d.t_ptr, d.t_col, d.t_thresh, val, term,
                                                   pref_c, pref_v, fin, enter))
      return;
  } else {
    if (!enter()) return;
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

// The Halpern variant's decision: every step is taken at the constant step size; the
// fixed-point residual r = ||z - T(z)||_P of this step, ||(dx, dy)||_P^2 =
// (omega / eta) ||dx||^2 + ||dy||^2 / (omega eta) - 2 dy^T K dx (scaled norms), is
// recorded for the restart rules (the epoch's first step also sets r_0) and in the
// decision trace (as eta_bar); then the Halpern coefficients of the next step.
template <typename T>
__device__ __forceinline__ void decide_halpern(DevState* st, T dx2, T dy2, T dkd) {
  constexpr bool F64 = std::is_same<T, double>::value;
  st->attempts += 1;
  if (!isfinite(dx2) || !isfinite(dy2) || !isfinite(dkd)) {
    st->status = 4;  // PDLP_NUMERICAL
    return;
  }
  const T eta = F64 ? (T)st->eta : (T)st->eta_f;
  const T om = F64 ? (T)st->omega : (T)st->omega_f;
  const T iom = F64 ? (T)st->inv_omega : (T)st->inv_omega_f;
  const T r2 = F64 ? om / eta * dx2 + dy2 / (om * eta) - (T)2 * dkd
                   : (om * dx2 + dy2 * iom) / eta - (T)2 * dkd;
  const double r = sqrt(fmax((double)r2, 0.0));
  st->h_res = r;
  if (st->h_k == 0) st->h_r0 = r;
  const long long t = st->attempts - 1;
  if (t < st->tr_cap) {
    st->tr_eta[t] = (double)eta;
    st->tr_eta_bar[t] = r;
    st->tr_accepted[t] = 1;
  }
  st->cur ^= 1;  // the current buffers hold T(z): the candidate of the checks
  st->iters += 1;
  if (st->iters % st->period == 0 || st->iters >= st->iter_limit) st->check_due = 1;
  st->h_k += 1;
  halpern_coeffs(st);
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
  g->h_k = l.h_k;
  g->h_res = l.h_res;
  g->h_r0 = l.h_r0;
  g->ha_d = l.ha_d;
  g->hb_d = l.hb_d;
  g->hc_d = l.hc_d;
  g->ha_f = l.ha_f;
  g->hb_f = l.hb_f;
  g->hc_f = l.hc_f;
}

// ---------------------------------------------------------------- A5 + A6: dual
template <int LANES, typename T, typename V, bool IMPLICIT, bool H = false>
__global__ void __launch_bounds__(kBlock, StepOcc<T>::value) k_dual(IterData<T, V> d) {
  constexpr bool TILED = std::is_same<T, double>::value;
  const Span sp = make_span(d.td, d.m, d.grid_d_short, d.a_long, d.a_nlong);
  DevState* st = d.st + sp.lp;
  const vec2_t<T>* xn = nullptr;
  const T* y = nullptr;
  T* yn = nullptr;
  T sigma = 0, pw = 0, ha = 0, hb = 0, hc = 0;
  auto enter = [&]() -> bool {
    pdl_enter();
    if (st->status != 0 || st->check_due) return false;
    const int cur = st->cur;
    xn = cur ? d.x[0] : d.x[1];
    y = cur ? d.y[1] : d.y[0];
    yn = cur ? d.y[0] : d.y[1];
    sigma = StepT<T>::sigma(st);
    if constexpr (H) {
      ha = StepT<T>::ha(st);
      hb = StepT<T>::hb(st);
      hc = StepT<T>::hc(st);
    } else {
      pw = StepT<T>::pw(st);
    }
    return true;
  };
  T dy2 = 0, dkd = 0;
  // acc.a = (K x')_i, acc.b = (K dx)_i
  auto val = [&](int p) -> T { return Ld<T, V>::get(d.a_val, p); };
  auto term = [&](T v, int j) -> P2<T> {
    const vec2_t<T> xv = xn[j];
    return P2<T>{v * xv.x, v * xv.y};
  };
  auto load = [&](int p) -> P2<T> { return term(val(p), __ldg(d.a_col + p)); };
  auto pref_c = [&](int i) -> PreCD<T> {
    return PreCD<T>{__ldg(d.q + i), IMPLICIT ? __ldg(d.sw + i) : (T)1, (int)__ldg(d.row_kind + i)};
  };
  auto pref_v = [&](int i) -> PreVD<T> {
    if constexpr (H) return PreVD<T>{d.hy[i], d.hay[i]};  // the iterate and its anchor
    return PreVD<T>{y[i], pw != (T)0 ? d.sum_y[i] : (T)0};
  };
  auto fin = [&](int i, P2<T> acc, const PreCD<T>& c, const PreVD<T>& v) {
    const T kxbar = acc.a + acc.b;  // K (2x' - x)
    const T step = IMPLICIT ? sigma * c.sw : sigma;
    T yv = v.yo + step * (c.q - kxbar);
    if (c.kind != 1) yv = maxv(yv, (T)0);
    yn[i] = yv;
    if constexpr (H)
      d.hy[i] = ha * yv + hb * v.yo + hc * v.sy;  // the reflected Halpern mix
    else if (pw != (T)0)
      d.sum_y[i] = v.sy + pw * v.yo;
    const T dd = yv - v.yo;
    dy2 += IMPLICIT ? dd * dd / c.sw : dd * dd;
    dkd += dd * acc.b;
  };
  auto epi = [&](int i, P2<T> acc) { fin(i, acc, pref_c(i), pref_v(i)); };
  if constexpr (TILED) {
    if (!enter()) return;
    rows_all<true, LANES, P2<T>>(sp, d.a_ptr, d.a_thresh, load, epi);
  } else if (sp.bidx < sp.nshort) {
    if (!rows_short3<LANES, P2<T>, PreCD<T>, PreVD<T>, true>(sp, d.a_ptr, d.a_col, d.a_thresh, val,
                                                             term, pref_c, pref_v, fin, enter))
      return;
  } else {
    if (!enter()) return;
    rows_long<P2<T>>(sp, d.a_ptr, load, epi);
  }
  const T s0 = block_sum1<T>(dy2);
  const T s1 = block_sum1<T>(dkd);
  if (threadIdx.x == 0) {
    d.part_d[blockIdx.x] = s0;
    d.part_d[d.grid_d + blockIdx.x] = s1;
  }
}

// ---------------------------------------------------------------- A6: decision
// One block per LP, launched after the dual kernel (programmatic dependent
// launch): the LP's partial sums of ||dx||^2, ||dy||^2 and dy^T K dx in the
// order of their slots, then the step decision.  The state was last written by
// the previous decision or KKT block, grids that completed before the primal
// and dual kernels of this attempt began, so it is copied to shared memory, and
// this attempt's step-rule factors looked up, BEFORE the wait; after it only
// the partial sums are read.  In dry mode (launch-shape tuning) nothing is
// decided.
template <typename T, typename V>
__global__ void __launch_bounds__(kBlock) k_decide(IterData<T, V> d) {
  __shared__ DevState ls;
  __shared__ T fac[2];
  const int k = blockIdx.x;
  DevState* st = d.st + k;
  if (threadIdx.x < 32) {  // warp 0 copies the state word by word
    static_assert(sizeof(DevState) % 8 == 0, "state copied in 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(st);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&ls);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / 8); w += 32) dst[w] = src[w];
    __syncwarp();
    if (threadIdx.x == 0) step_factors(&ls, ls.attempts + 1, &fac[0], &fac[1]);
  }
  int p0 = 0, pn = d.grid_p, q0 = 0, qn = d.grid_d;
  if (d.tp.blk_lp != nullptr) {
    p0 = d.tp.blk0[k];
    pn = d.tp.nblk[k];
    q0 = d.td.blk0[k];
    qn = d.td.nblk[k];
  }
  __syncthreads();
  pdl_enter();
  if (ls.status != 0 || ls.check_due || ls.dry) {
    // inside a graph's while loop: nothing left to step in this check period
    if (d.cond && k == 0 && threadIdx.x == 0) cudaGraphSetConditional(d.cond, 0u);
    return;
  }
  T a = 0, b0 = 0, b1 = 0;
  if (std::is_same<T, float>::value && d.tile) {
    // tile kernels: one slot per (worker, LP) run -- the LP's first min(items, workers)
    // item slots, tslot entries each -- and one per long row
    const int i0 = d.tt.item0[k], i1 = min(d.tt.item0[k + 1], i0 + d.work_tt);
    for (int i = i0 * d.tslot + threadIdx.x; i < i1 * d.tslot; i += kBlock) a += (T)d.tt.part[i].x;
    for (int i = d.tt.lng0[k] + threadIdx.x; i < d.tt.lng0[k + 1]; i += kBlock) a += (T)d.tt.lterm[i].x;
    const int j0 = d.ta.item0[k], j1 = min(d.ta.item0[k + 1], j0 + d.work_ta);
    for (int i = j0 * d.tslot + threadIdx.x; i < j1 * d.tslot; i += kBlock) {
      const float2 v = d.ta.part[i];
      b0 += (T)v.x;
      b1 += (T)v.y;
    }
    for (int i = d.ta.lng0[k] + threadIdx.x; i < d.ta.lng0[k + 1]; i += kBlock) {
      const float2 v = d.ta.lterm[i];
      b0 += (T)v.x;
      b1 += (T)v.y;
    }
  } else {
    for (int i = threadIdx.x; i < pn; i += kBlock) a += d.part_p[p0 + i];
    for (int i = threadIdx.x; i < qn; i += kBlock) {
      b0 += d.part_d[q0 + i];
      b1 += d.part_d[d.grid_d + q0 + i];
    }
  }
  block_sum3<T>(a, b0, b1);
  if (threadIdx.x == 0) {
    if (ls.halpern)
      decide_halpern<T>(&ls, a, b0, b1);
    else
      decide_step<T>(&ls, a, b0, b1, fac[0], fac[1]);
    store_step_state(st, ls);
    if (d.cond && k == 0) {
      // one LP in a graph with a while loop: keep stepping until a KKT check falls
      // due, the solve stops, or this graph launch has run loop_cap attempts
      const int la = ls.loop_attempts + 1;
      st->loop_attempts = la;
      cudaGraphSetConditional(d.cond,
                              (ls.status == 0 && !ls.check_due && la < d.loop_cap) ? 1u : 0u);
    }
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
// (y in the primal phase, the (x', dx) pairs in the dual phase) are read with
// ordinary loads, which each grid barrier orders after the writes (thread 0's
// acquire load of the barrier generation, after the writers' fence and arrival,
// then a block barrier); the partial sums are read through L2 (ld.global.cg);
// nothing the kernel writes goes through the non-coherent read-only path.  The
// float32 phases use the pipelined row traversal of the two-launch kernels.
// Partial sums alternate between two buffers by attempt parity, so a block
// still reducing attempt k never sees attempt k + 1's values.  Every barrier
// wait is bounded: a block that gives up flags the
// state (kStatusWaitFailed) and returns, and so do the others.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_barrier(DevState* st) {
  if (gridDim.x == 1) {  // a one-block launch: the block's barrier orders its global memory
    __syncthreads();
    return true;
  }
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(&st->bar_gen);
    __threadfence();
    int good = 1;
    const long long limit = st->spin_limit;
    // a skipped arrival (fault-handling tests) leaves every block waiting until its limit
    const bool arrive = !(st->bar_skip && blockIdx.x == 0);
    if (arrive && atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      long long polls = 0;
      while (ld_acquire_u32(&st->bar_gen) == gen) {
        if (++polls > limit || *(volatile int*)&st->bar_err) {
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

// The persistent kernel over a batch (persistent = 1 with count > 1): the resident grid
// walks the two launch maps' virtual blocks (block b takes b, b + G, ...; each virtual
// block belongs to one LP and keeps its rows and its partial-sum slot, as in the
// two-launch form), with three grid barriers per attempt: after the primal phase, after
// the dual phase, and after the decisions, which block b takes for the LPs b, b + G, ...
// from the LP's slots in order.  Each LP steps until its own check falls due or it
// stops; the launch ends when no LP steps any more or after `max_attempts`.  The state
// and the partial sums are read through L2; vector entries other blocks wrote in an earlier
// phase are read with ordinary loads: each grid barrier ends with thread 0's acquire load of
// the barrier generation (after the writers' fence and arrival) and a block barrier, which
// orders them after those writes.  The float32 phases use the same pipelined row traversal
// as the two-launch kernels.
template <typename T>
struct StepView {
  int go, cur;
  T tau, sigma, pw;
};
template <typename T>
__device__ __forceinline__ StepView<T> step_view(const DevState* st) {
  StepView<T> v;
  v.go = __ldcg(&st->status) == 0 && __ldcg(&st->check_due) == 0;
  v.cur = __ldcg(&st->cur);
  if constexpr (std::is_same<T, float>::value) {
    v.tau = __ldcg(&st->tau_f);
    v.sigma = __ldcg(&st->sigma_f);
    v.pw = __ldcg(&st->pw_f);
  } else {
    v.tau = __ldcg(&st->tau_d);
    v.sigma = __ldcg(&st->sigma_d);
    v.pw = __ldcg(&st->pending_w);
  }
  return v;
}

template <int LA, int LT, typename T, typename V, bool IMPLICIT>
__device__ __forceinline__ void persist_batch(const IterData<T, V>& d, int max_attempts) {
  constexpr bool TILED = std::is_same<T, double>::value;
  DevState* gst = d.st;  // LP 0's state also holds the grid barrier's words
  const int G = gridDim.x, b = blockIdx.x;
  __shared__ StepView<T> vsh;
  __shared__ DevState ls;
  __shared__ T fac[2];
  __shared__ int go_any;
  for (int att = 0; att < max_attempts; ++att) {
    // ---- A4: primal phase over the virtual blocks of the A^T map
    for (int vb = b; vb < d.grid_p; vb += G) {
      const Span sp = span_of(d.tp, vb, d.t_long);
      if (threadIdx.x == 0) vsh = step_view<T>(d.st + sp.lp);
      __syncthreads();
      const StepView<T> v = vsh;
      __syncthreads();
      if (!v.go) continue;
      const vec2_t<T>* x = v.cur ? d.x[1] : d.x[0];
      vec2_t<T>* xn = v.cur ? d.x[0] : d.x[1];
      const T* y = v.cur ? d.y[1] : d.y[0];
      T dx2 = 0;
      auto val = [&](int p) -> T { return Ld<T, V>::get(d.t_val, p); };
      auto term = [&](T a, int i) -> T { return a * y[i]; };
      auto load = [&](int p) -> T { return term(val(p), __ldg(d.t_col + p)); };
      auto pref_c = [&](int j) -> PreCP<T> {
        return PreCP<T>{__ldg(d.c + j), __ldg(d.l + j), __ldg(d.u + j),
                        IMPLICIT ? __ldg(d.tw + j) : (T)1};
      };
      auto pref_v = [&](int j) -> PreVP<T> {
        return PreVP<T>{x[j].x, v.pw != (T)0 ? d.sum_x[j] : (T)0};
      };
      auto fin = [&](int j, T aty, const PreCP<T>& c, const PreVP<T>& pv) {
        const T step = IMPLICIT ? v.tau * c.tw : v.tau;
        const T xv = clampv(pv.xo - step * (c.c - aty), c.l, c.u);
        const T dd = xv - pv.xo;
        vec2_t<T> o;
        o.x = xv;
        o.y = dd;
        xn[j] = o;
        if (v.pw != (T)0) d.sum_x[j] = pv.sx + v.pw * pv.xo;
        dx2 += IMPLICIT ? dd * dd / c.tw : dd * dd;
      };
      auto epi = [&](int j, T aty) { fin(j, aty, pref_c(j), pref_v(j)); };
      if constexpr (TILED) {
        rows_all<true, LT, T>(sp, d.t_ptr, d.t_thresh, load, epi);
      } else if (sp.bidx < sp.nshort) {
        rows_short3<LT, T, PreCP<T>, PreVP<T>>(sp, d.t_ptr, d.t_col, d.t_thresh, val, term, pref_c,
                                               pref_v, fin, [] { return true; });
      } else {
        rows_long<T>(sp, d.t_ptr, load, epi);
      }
      const T s = block_sum1<T>(dx2);
      if (threadIdx.x == 0) d.part_p[vb] = s;
    }
    if (!grid_barrier(gst)) return;
    // ---- A5: dual phase over the virtual blocks of the A map
    for (int vb = b; vb < d.grid_d; vb += G) {
      const Span sp = span_of(d.td, vb, d.a_long);
      if (threadIdx.x == 0) vsh = step_view<T>(d.st + sp.lp);
      __syncthreads();
      const StepView<T> v = vsh;
      __syncthreads();
      if (!v.go) continue;
      const vec2_t<T>* xn = v.cur ? d.x[0] : d.x[1];
      const T* y = v.cur ? d.y[1] : d.y[0];
      T* yn = v.cur ? d.y[0] : d.y[1];
      T dy2 = 0, dkd = 0;
      auto val = [&](int p) -> T { return Ld<T, V>::get(d.a_val, p); };
      auto term = [&](T a, int j) -> P2<T> {
        const vec2_t<T> xv = xn[j];
        return P2<T>{a * xv.x, a * xv.y};
      };
      auto load = [&](int p) -> P2<T> { return term(val(p), __ldg(d.a_col + p)); };
      auto pref_c = [&](int i) -> PreCD<T> {
        return PreCD<T>{__ldg(d.q + i), IMPLICIT ? __ldg(d.sw + i) : (T)1, (int)__ldg(d.row_kind + i)};
      };
      auto pref_v = [&](int i) -> PreVD<T> {
        return PreVD<T>{y[i], v.pw != (T)0 ? d.sum_y[i] : (T)0};
      };
      auto fin = [&](int i, P2<T> acc, const PreCD<T>& c, const PreVD<T>& pv) {
        const T step = IMPLICIT ? v.sigma * c.sw : v.sigma;
        T yv = pv.yo + step * (c.q - (acc.a + acc.b));
        if (c.kind != 1) yv = maxv(yv, (T)0);
        yn[i] = yv;
        if (v.pw != (T)0) d.sum_y[i] = pv.sy + v.pw * pv.yo;
        const T dd = yv - pv.yo;
        dy2 += IMPLICIT ? dd * dd / c.sw : dd * dd;
        dkd += dd * acc.b;
      };
      auto epi = [&](int i, P2<T> acc) { fin(i, acc, pref_c(i), pref_v(i)); };
      if constexpr (TILED) {
        rows_all<true, LA, P2<T>>(sp, d.a_ptr, d.a_thresh, load, epi);
      } else if (sp.bidx < sp.nshort) {
        rows_short3<LA, P2<T>, PreCD<T>, PreVD<T>>(sp, d.a_ptr, d.a_col, d.a_thresh, val, term,
                                                   pref_c, pref_v, fin, [] { return true; });
      } else {
        rows_long<P2<T>>(sp, d.a_ptr, load, epi);
      }
      const T s0 = block_sum1<T>(dy2);
      const T s1 = block_sum1<T>(dkd);
      if (threadIdx.x == 0) {
        d.part_d[vb] = s0;
        d.part_d[d.grid_d + vb] = s1;
      }
    }
    if (!grid_barrier(gst)) return;
    // ---- A6: the decisions, block b for the LPs b, b + G, ...
    for (int k = b; k < d.count; k += G) {
      if (threadIdx.x < 32) {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(d.st + k);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&ls);
        for (int w = threadIdx.x; w < (int)(sizeof(DevState) / 8); w += 32) dst[w] = __ldcg(src + w);
        __syncwarp();
        if (threadIdx.x == 0) step_factors(&ls, ls.attempts + 1, &fac[0], &fac[1]);
      }
      __syncthreads();
      if (ls.status == 0 && !ls.check_due && !ls.dry) {
        const int p0 = d.tp.blk0[k], pn = d.tp.nblk[k], q0 = d.td.blk0[k], qn = d.td.nblk[k];
        T a = 0, b0 = 0, b1 = 0;
        for (int i = threadIdx.x; i < pn; i += kBlock) a += __ldcg(d.part_p + p0 + i);
        for (int i = threadIdx.x; i < qn; i += kBlock) {
          b0 += __ldcg(d.part_d + q0 + i);
          b1 += __ldcg(d.part_d + d.grid_d + q0 + i);
        }
        block_sum3<T>(a, b0, b1);
        if (threadIdx.x == 0) {
          decide_step<T>(&ls, a, b0, b1, fac[0], fac[1]);
          store_step_state(d.st + k, ls);
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(gst)) return;
    // ---- does any LP still step?  (every block reads the same states)
    int mine = 0;
    for (int k = threadIdx.x; k < d.count; k += kBlock)
      mine |= __ldcg(&d.st[k].status) == 0 && __ldcg(&d.st[k].check_due) == 0;
    if (threadIdx.x == 0) go_any = 0;
    __syncthreads();
    if (mine) go_any = 1;
    __syncthreads();
    if (!go_any) break;
  }
}

template <int LA, int LT, typename T, typename V, bool IMPLICIT>
__global__ void __launch_bounds__(kBlock) k_persist(IterData<T, V> d, int max_attempts) {
  constexpr bool TILED = std::is_same<T, double>::value;
  if (d.tp.blk_lp != nullptr) {  // a batch
    persist_batch<LA, LT, T, V, IMPLICIT>(d, max_attempts);
    return;
  }
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
      auto val = [&](int p) -> T { return Ld<T, V>::get(d.t_val, p); };
      auto term = [&](T a, int i) -> T { return a * y[i]; };
      auto load = [&](int p) -> T { return term(val(p), __ldg(d.t_col + p)); };
      auto pref_c = [&](int j) -> PreCP<T> {
        return PreCP<T>{__ldg(d.c + j), __ldg(d.l + j), __ldg(d.u + j),
                        IMPLICIT ? __ldg(d.tw + j) : (T)1};
      };
      auto pref_v = [&](int j) -> PreVP<T> {
        return PreVP<T>{x[j].x, pw != (T)0 ? d.sum_x[j] : (T)0};
      };
      auto fin = [&](int j, T aty, const PreCP<T>& c, const PreVP<T>& pv) {
        const T step = IMPLICIT ? tau * c.tw : tau;
        const T xv = clampv(pv.xo - step * (c.c - aty), c.l, c.u);
        const T dd = xv - pv.xo;
        vec2_t<T> o;
        o.x = xv;
        o.y = dd;
        xn[j] = o;
        if (pw != (T)0) d.sum_x[j] = pv.sx + pw * pv.xo;
        dx2 += IMPLICIT ? dd * dd / c.tw : dd * dd;
      };
      auto epi = [&](int j, T aty) { fin(j, aty, pref_c(j), pref_v(j)); };
      if constexpr (TILED)
        rows_tiled<LT, T>(sp_p, d.t_ptr, d.t_thresh, load, epi);
      else
        rows_short3<LT, T, PreCP<T>, PreVP<T>>(sp_p, d.t_ptr, d.t_col, d.t_thresh, val, term,
                                               pref_c, pref_v, fin, [] { return true; });
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
      auto val = [&](int p) -> T { return Ld<T, V>::get(d.a_val, p); };
      auto term = [&](T a, int j) -> P2<T> {
        const vec2_t<T> xv = xn[j];
        return P2<T>{a * xv.x, a * xv.y};
      };
      auto load = [&](int p) -> P2<T> { return term(val(p), __ldg(d.a_col + p)); };
      auto pref_c = [&](int i) -> PreCD<T> {
        return PreCD<T>{__ldg(d.q + i), IMPLICIT ? __ldg(d.sw + i) : (T)1, (int)__ldg(d.row_kind + i)};
      };
      auto pref_v = [&](int i) -> PreVD<T> {
        return PreVD<T>{y[i], pw != (T)0 ? d.sum_y[i] : (T)0};
      };
      auto fin = [&](int i, P2<T> acc, const PreCD<T>& c, const PreVD<T>& pv) {
        const T step = IMPLICIT ? sigma * c.sw : sigma;
        T yv = pv.yo + step * (c.q - (acc.a + acc.b));
        if (c.kind != 1) yv = maxv(yv, (T)0);
        yn[i] = yv;
        if (pw != (T)0) d.sum_y[i] = pv.sy + pw * pv.yo;
        const T dd = yv - pv.yo;
        dy2 += IMPLICIT ? dd * dd / c.sw : dd * dd;
        dkd += dd * acc.b;
      };
      auto epi = [&](int i, P2<T> acc) { fin(i, acc, pref_c(i), pref_v(i)); };
      if constexpr (TILED)
        rows_tiled<LA, P2<T>>(sp_d, d.a_ptr, d.a_thresh, load, epi);
      else
        rows_short3<LA, P2<T>, PreCD<T>, PreVD<T>>(sp_d, d.a_ptr, d.a_col, d.a_thresh, val, term,
                                                   pref_c, pref_v, fin, [] { return true; });
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
