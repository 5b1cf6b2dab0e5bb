// KKT evaluation, restart decision and primal-weight update (rows A8-A10),
// all in float64 on the unscaled canonical data, run once per check period.
//
//   k_kkt_prep   unscaled float64 current iterate and step-size-weighted
//                average (A7) into scratch vectors; with the certificate test
//                on, also the rays x^ = x - x_last projected onto the recession
//                cone of [l, u] and y^ = y - y_last projected onto Y
//   k_kkt_rows   K x for both candidates in one pass over A, fused with the
//                primal residuals (unscaled and scaled), q^T y and the scaled
//                dual distance to the last restart point
//   k_kkt_cols   K^T y for both candidates in one pass over A^T, fused with
//                the bound-aware dual residuals, objective terms and the scaled
//                primal distance to the last restart point
//   k_kkt_final  one block: fixed-order reduction of the partials, relative
//                KKT of both candidates (the termination test of the paper's
//                relative tolerances, section 4), the certificates of primal
//                and dual infeasibility, the KKT restart criteria and the
//                primal-weight update
//   k_kkt_apply  restart: replace the iterate by the average if chosen, move
//                the restart anchors, clear the running sums
//   k_kkt_end    one thread: clear the per-check flags
#include "internal.h"
#include "iter_kernels.cuh"

namespace pdlp {

namespace {

// weighted average sum / sw: a division for float64 iterates (the parity mode
// divides where the definition divides), the block's reciprocal otherwise
#define avg_of(sum, sw, isw) (std::is_same<T, double>::value ? (sum) / (sw) : (sum) * (isw))

// (current, average) of a candidate entry: one 16-byte load (ordinary loads: the
// vectors are written by the preceding kernel of the same chain)
__device__ __forceinline__ double2 cand2(const double2* g, long long i) { return g[i]; }

// columns and rows of one LP for the elementwise kernels (prep, apply, output)
struct ESpan {
  int lp, c0, nc, r0, nr, bidx, nblk;
};
__device__ __forceinline__ ESpan make_espan(const KktRaw& r) {
  if (r.tc.blk_lp == nullptr) return ESpan{0, 0, r.n, 0, r.m, (int)blockIdx.x, (int)gridDim.x};
  const int k = r.tc.blk_lp[blockIdx.x];
  return ESpan{k, r.tc.row0[k], r.tc.nrows[k], r.tr.row0[k], r.tr.nrows[k],
               (int)blockIdx.x - r.tc.blk0[k], r.tc.nblk[k]};
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_kkt_prep(KktRaw r) {
  pdl_enter();
  const ESpan es = make_espan(r);
  DevState* st = r.st + es.lp;
  if (!st->check_due || st->status != 0) return;
  const int cur = st->cur;
  const double pw = st->pending_w, sw = st->sum_w;
  const vec2_t<T>* x = (const vec2_t<T>*)r.x[cur];
  const T* y = (const T*)r.y[cur];
  const T* sx = (const T*)r.sum_x;
  const T* sy = (const T*)r.sum_y;
  __shared__ double inv_sh;  // one float64 division per block, not per element
  if (threadIdx.x == 0) inv_sh = sw > 0.0 ? 1.0 / sw : 0.0;
  __syncthreads();
  const double isw = inv_sh;
  const long long stride = (long long)es.nblk * kBlock;
  for (long long j = es.c0 + (long long)es.bidx * kBlock + threadIdx.x; j < es.c0 + es.nc; j += stride) {
    const double xc = (double)x[j].x;
    const double xa = sw > 0.0 ? avg_of((double)sx[j] + pw * xc, sw, isw) : xc;
    const double s = r.scaled ? r.dc[j] : r.ux;
    // unscaled candidates, clipped to [l, u] so the KKT measured here is the
    // KKT of exactly the point the solver returns (A11)
    const double Xc = fmin(fmax(s * xc, r.l[j]), r.u[j]);
    double d = 0.0;
    if (r.rays == 2) {
      // displacement since the restart anchor, on the recession cone of [l, u]
      const unsigned f = r.bflags[j];
      d = Xc - r.Xl[j];
      if (f & 1u) d = fmax(d, 0.0);
      if (f & 2u) d = fmin(d, 0.0);
    }
    r.XG[j] = make_double2(Xc, fmin(fmax(s * xa, r.l[j]), r.u[j]));
    if (r.rays == 2) r.XR[j] = d;
    if (r.chk_pts && !st->init_pending)  // row (completed checks) mod capacity
      r.chk_pts[(size_t)(st->checks % r.chk_cap) * (size_t)r.n + (size_t)j] = Xc;
  }
  for (long long i = es.r0 + (long long)es.bidx * kBlock + threadIdx.x; i < es.r0 + es.nr; i += stride) {
    const double yc = (double)y[i];
    const double ya = sw > 0.0 ? avg_of((double)sy[i] + pw * yc, sw, isw) : yc;
    const double s = r.scaled ? r.dr[i] : r.uy;
    const double Yc = s * yc;
    double d = 0.0;
    if (r.rays) {
      d = Yc - r.Yl[i];
      if (r.row_kind[i] != 1) d = fmax(d, 0.0);
    }
    r.YG[i] = make_double2(Yc, s * ya);
    if (r.rays) r.YR[i] = d;
  }
}

// partial layout over rows of A: [0,1] ||r_p||^2 cur/avg, [2,3] ||D_r r_p||^2,
// [4,5] q^T y, [6,7] ||(y - y_last) / D_r||^2; with RAYS >= 1 also [9] q^T y^ and
// [10] sum |q_i y^_i| of the dual ray, with RAYS = 2 [8] ||r^_p||^2 of the primal ray
// (RAYS = 1 when every column is boxed: the primal ray is 0 and [8] stays 0)
template <int LANES, int RAYS>
__global__ void __launch_bounds__(kBlock) k_kkt_rows(KktRaw r) {
  pdl_enter();
  const Span sp = make_span(r.tr, r.m, r.grid_r_short, r.a_long, r.a_nlong);
  DevState* st = r.st + sp.lp;
  if (!st->check_due || st->status != 0) return;
  constexpr int NV = RAYS ? 11 : 8;
  using Acc = typename std::conditional<RAYS == 2, D3, D2>::type;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  const double* __restrict__ val = r.a_val64;
  auto load = [&](int p) -> Acc {
    const double v = val ? __ldg(val + p) : 1.0;
    const int j = __ldg(r.a_col + p);
    const double2 x2 = cand2(r.XG, j);
    if constexpr (RAYS == 2)
      return D3{v * x2.x, v * x2.y, v * r.XR[j]};
    else
      return D2{v * x2.x, v * x2.y};
  };
  auto epi = [&](int i, Acc ax) {
    const double q = r.q[i], dr = r.dr[i];
    const bool eq = r.row_kind[i] == 1;
    const double kx[2] = {ax.a, ax.b};
    const double2 y2 = cand2(r.YG, i);
    const double yv[2] = {y2.x, y2.y};
    // A9b: D_r times the scaled gap gradient q~ - K~ x~ = D_r (q - K x) of both candidates
    if (r.ndg_gy) r.ndg_gy[i] = make_double2(dr * (dr * (q - kx[0])), dr * (dr * (q - kx[1])));
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      double rp = q - kx[k];
      if (!eq) rp = fmax(rp, 0.0);
      acc[0 + k] += rp * rp;
      acc[2 + k] += (dr * rp) * (dr * rp);
      acc[4 + k] += q * yv[k];
      const double dd = (yv[k] - r.Yl[i]) * r.inv_dr[i];
      acc[6 + k] += dd * dd;
    }
    if constexpr (RAYS == 2) {
      // A12: the primal ray must keep K x^ >= 0 (= 0 on equality rows)
      const double rr = eq ? fabs(ax.c) : fmax(-ax.c, 0.0);
      acc[8] += rr * rr;
    }
    if constexpr (RAYS >= 1) {
      const double qy = q * r.YR[i];
      acc[9] += qy;
      acc[10] += fabs(qy);
    }
  };
  rows_all<true, LANES, Acc>(sp, r.a_ptr, r.a_thresh, load, epi);
  double out[NV];
  block_sum_rs<NV>(acc, out);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) r.part_r[(size_t)k * r.grid_r + blockIdx.x] = out[k];
}

// partial layout over rows of A^T: [0,1] ||r_d||^2, [2,3] ||D_c r_d||^2, [4,5] c^T x,
// [6,7] bound terms of the dual objective, [8,9] ||(x - x_last) / D_c||^2; with
// RAYS >= 1 also, for the dual ray (lambda^ = -K^T y^): [11] its bound terms,
// [12] their magnitudes; with RAYS = 2 [10] ||r^_d||^2 and for the primal ray
// [13] c^T x^, [14] sum |c_j x^_j| (all 0 when every column is boxed)
template <int LANES, int RAYS>
__global__ void __launch_bounds__(kBlock) k_kkt_cols(KktRaw r) {
  pdl_enter();
  const Span sp = make_span(r.tc, r.n, r.grid_c_short, r.t_long, r.t_nlong);
  DevState* st = r.st + sp.lp;
  if (!st->check_due || st->status != 0) return;
  constexpr int NV = RAYS ? 15 : 10;
  using Acc = typename std::conditional<RAYS, D3, D2>::type;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  const double* __restrict__ val = r.t_val64;
  auto load = [&](int p) -> Acc {
    const double v = val ? __ldg(val + p) : 1.0;
    const int i = __ldg(r.t_col + p);
    const double2 y2 = cand2(r.YG, i);
    if constexpr (RAYS)
      return D3{v * y2.x, v * y2.y, v * r.YR[i]};
    else
      return D2{v * y2.x, v * y2.y};
  };
  auto epi = [&](int j, Acc aty) {
    const double c = r.c[j], dc = r.dc[j], idc = r.inv_dc[j];
    const unsigned f = r.bflags[j];
    const bool lfin = f & 1u, ufin = f & 2u;
    const double l = lfin ? r.l[j] : 0.0, u = ufin ? r.u[j] : 0.0;
    const double kty[2] = {aty.a, aty.b};
    const double2 x2 = cand2(r.XG, j);
    const double xv[2] = {x2.x, x2.y};
    // A9b: D_c times the scaled gap gradient K~^T y~ - c~ = D_c (K^T y - c)
    if (r.ndg_gx) r.ndg_gx[j] = make_double2(dc * (dc * (kty[0] - c)), dc * (dc * (kty[1] - c)));
    // lambda+ = lam, lambda- = 0 when lam > 0, else lambda+ = 0, lambda- = -lam: each
    // term below keeps only its nonzero part (the same values; the sign test is an
    // integer compare, so the float64 pipe does the arithmetic only)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double lam = c - kty[k];
      const bool pos = __double_as_longlong(lam) > 0;
      const double rd = pos ? (lfin ? 0.0 : lam) : (ufin ? 0.0 : -lam);
      acc[0 + k] += rd * rd;
      acc[2 + k] += (dc * rd) * (dc * rd);
      acc[4 + k] += c * xv[k];
      acc[6 + k] += (pos ? l : u) * lam;  // l lambda+ - u lambda-; l, u read as 0 where infinite
      const double dd = (xv[k] - r.Xl[j]) * idc;
      acc[8 + k] += dd * dd;
    }
    if constexpr (RAYS >= 1) {
      // A12: the dual ray's reduced cost has no c
      const double lam = -aty.c;
      const bool pos = __double_as_longlong(lam) > 0;
      const double t = (pos ? l : u) * lam;
      acc[11] += t;
      acc[12] += fabs(t);
      if constexpr (RAYS == 2) {
        const double rd = pos ? (lfin ? 0.0 : lam) : (ufin ? 0.0 : -lam);
        acc[10] += rd * rd;
        const double cx = c * r.XR[j];
        acc[13] += cx;
        acc[14] += fabs(cx);
      }
    }
  };
  rows_all<true, LANES, Acc>(sp, r.t_ptr, r.t_thresh, load, epi);
  double out[NV];
  block_sum_rs<NV>(acc, out);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) r.part_c[(size_t)k * r.grid_c + blockIdx.x] = out[k];
}

// A12: a ray whose objective `obj` (oriented so that a certificate has obj > 0)
// clears the rounding of its terms (`mag`, the sum of their magnitudes) and whose
// residual is within eps_inf of it
__device__ __forceinline__ bool inf_certificate(double obj, double mag, double res) {
  constexpr double eps_inf = 1e-8, kappa = 1e-9;
  return obj > 0.0 && obj > kappa * mag && res <= eps_inf * obj;
}

// A9b: one stage of the normalized duality gaps of both candidates (current, average)
// at a check, in scaled space through the unscaled candidates X = D_c x~, Y = D_r y~:
// for the trial steps t of the two candidates every block adds, over its columns and
// rows, the squared omega-distance of z^(t) = (proj_[l,u](X + (t / omega) D_c g~_x),
// proj_Y(Y + t omega D_r g~_y)) from z and the gap g~^T (z~^(t) - z~) (stage 0: the
// squared radius from the last restart point and the squared dual norm N^2 =
// ||g~_x||^2 / omega + omega ||g~_y||^2); the last block to finish adds the blocks'
// partials in slot order and advances both candidates' bisection.  One LP.
__device__ void ndg_advance(NdgState* g, const double* sum) {
  const int stage = g->stage;
  for (int c = 0; c < 2; ++c) {
    NdgCand& k = g->c[c];
    if (stage == 0) {
      k.done = 0;
      k.fixed = 0;
      k.r = sqrt(sum[c]);
      k.nrm = sqrt(sum[2 + c]);
      k.rho = 0.0;
      if (k.r == 0.0 || k.nrm == 0.0) {
        k.done = 1;
        continue;
      }
      k.t0 = k.r / k.nrm;
      k.trial = ldexp(k.t0, 63);
      continue;
    }
    if (k.done) continue;
    const double d = sqrt(sum[c]);
    if (stage == 1) {
      if (d < k.r) {
        k.fixed = 1;  // the far end t0 2^63 is inside the ball: t stays there
      } else {
        k.lo = -1;
        k.hi = 63;
        k.mid = (k.lo + k.hi) >> 1;
        k.trial = ldexp(k.t0, k.mid);
      }
    } else if (stage < 2 + kNdgKSteps) {
      if (k.fixed) continue;
      if (d >= k.r) k.hi = k.mid; else k.lo = k.mid;
      if (stage == 1 + kNdgKSteps) {
        k.a = ldexp(k.t0, k.hi - 1);
        k.b = ldexp(k.t0, k.hi);
        k.trial = 0.5 * (k.a + k.b);
      } else {
        k.mid = (k.lo + k.hi) >> 1;  // floor, also for lo = -1
        k.trial = ldexp(k.t0, k.mid);
      }
    } else if (stage < 2 + kNdgKSteps + kNdgHalvings) {
      if (k.fixed) continue;
      if (d >= k.r) k.b = k.trial; else k.a = k.trial;
      k.trial = stage == 1 + kNdgKSteps + kNdgHalvings ? k.a : 0.5 * (k.a + k.b);
    } else {
      k.rho = sum[2 + c] / k.r;  // the gap at the final step over the radius
      k.done = 1;
    }
  }
  g->stage = stage + 1;
}

// one stage's partials of this thread over its columns and rows (strided by `stride`
// from `first`): stage 0 the squared radii and dual norms, later the squared distances
// and the gaps at the trial steps s0, s1
__device__ __forceinline__ void ndg_stage_sums(const KktRaw& r, int stage, double om, double iom,
                                               double s0, double s1, long long first,
                                               long long stride, double (&acc)[4]) {
  for (long long j = first; j < r.n; j += stride) {
    const double2 X = r.XG[j], D = r.ndg_gx[j];
    const double idc = r.inv_dc[j];
    if (stage == 0) {
      const double xl = r.Xl[j];
      const double d0 = (X.x - xl) * idc, d1 = (X.y - xl) * idc;
      acc[0] += om * d0 * d0;
      acc[1] += om * d1 * d1;
      const double g0 = D.x * idc, g1 = D.y * idc;
      acc[2] += g0 * g0 * iom;
      acc[3] += g1 * g1 * iom;
    } else {
      const double l = r.l[j], u = r.u[j];
      const double d0 = (fmin(fmax(X.x + (s0 * iom) * D.x, l), u) - X.x) * idc;
      const double d1 = (fmin(fmax(X.y + (s1 * iom) * D.y, l), u) - X.y) * idc;
      acc[0] += om * d0 * d0;
      acc[1] += om * d1 * d1;
      acc[2] += (D.x * idc) * d0;
      acc[3] += (D.y * idc) * d1;
    }
  }
  for (long long i = first; i < r.m; i += stride) {
    const double2 Y = r.YG[i], E = r.ndg_gy[i];
    const double idr = r.inv_dr[i];
    if (stage == 0) {
      const double yl = r.Yl[i];
      const double d0 = (Y.x - yl) * idr, d1 = (Y.y - yl) * idr;
      acc[0] += d0 * d0 * iom;
      acc[1] += d1 * d1 * iom;
      const double g0 = E.x * idr, g1 = E.y * idr;
      acc[2] += om * g0 * g0;
      acc[3] += om * g1 * g1;
    } else {
      const bool eq = r.row_kind[i] == 1;
      double y0 = Y.x + (s0 * om) * E.x, y1 = Y.y + (s1 * om) * E.y;
      if (!eq) {
        y0 = fmax(y0, 0.0);
        y1 = fmax(y1, 0.0);
      }
      const double d0 = (y0 - Y.x) * idr, d1 = (y1 - Y.y) * idr;
      acc[0] += d0 * d0 * iom;
      acc[1] += d1 * d1 * iom;
      acc[2] += (E.x * idr) * d0;
      acc[3] += (E.y * idr) * d1;
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_ndg_eval(KktRaw r) {
  pdl_enter();
  DevState* st = r.st;
  if (!st->check_due || st->status != 0 || st->init_pending) return;
  NdgState* g = r.ndg;
  const int stage = g->stage;  // the same in every block: written by an earlier launch
  if (stage >= kNdgStages) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  ndg_stage_sums(r, stage, st->omega, st->inv_omega, g->c[0].trial, g->c[1].trial,
                 (long long)blockIdx.x * kBlock + threadIdx.x, (long long)gridDim.x * kBlock,
                 acc);
  double out[4];
  block_sum_rs<4>(acc, out);
  __shared__ int last;
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) r.ndg_part[(size_t)k * gridDim.x + blockIdx.x] = out[k];
    __threadfence();
    last = atomicAdd(&g->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last block: every thread adds a strided share of the partials (read through L2),
  // then the block's fixed-order reduction
  __threadfence();
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kBlock)
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] += __ldcg(r.ndg_part + (size_t)k * gridDim.x + b);
  double sum[4];
  block_sum_rs<4>(v, sum);
  if (threadIdx.x != 0) return;
  g->ticket = 0;
  ndg_advance(g, sum);
}

// All the stages in one block (small LPs: n + m <= kNdgOneBlock), the block's reduction
// in place of the last-block hand-over; the same partial sums in the same order per
// thread, added in another order than k_ndg_eval's.
__global__ void __launch_bounds__(kBlock) k_ndg_block(KktRaw r) {
  pdl_enter();
  DevState* st = r.st;
  if (!st->check_due || st->status != 0 || st->init_pending) return;
  NdgState* g = r.ndg;
  const double om = st->omega, iom = st->inv_omega;
  for (int stage = 0; stage < kNdgStages; ++stage) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    ndg_stage_sums(r, stage, om, iom, g->c[0].trial, g->c[1].trial, threadIdx.x, kBlock, acc);
    double sum[4];
    block_sum_rs<4>(acc, sum);  // ends with a block barrier
    if (threadIdx.x == 0) ndg_advance(g, sum);
    __syncthreads();  // the next trial steps, written by thread 0
  }
}

__global__ void __launch_bounds__(kBlock) k_kkt_final(KktRaw r) {
  pdl_enter();
  // one block per LP
  const int k = blockIdx.x;
  DevState* st = r.st + k;
  if (!st->check_due || st->status != 0) return;
  int r0 = 0, rn = r.grid_r, c0 = 0, cn = r.grid_c;
  if (r.tr.blk_lp != nullptr) {
    r0 = r.tr.blk0[k];
    rn = r.tr.nblk[k];
    c0 = r.tc.blk0[k];
    cn = r.tc.nblk[k];
  }
  double pr[kPartR], pc[kPartC];
  if (r.rays) {
    reduce_partials<kPartR>(r.part_r + r0, r.grid_r, rn, pr);
    reduce_partials<kPartC>(r.part_c + c0, r.grid_c, cn, pc);
  } else {
    double a[8], b[10];
    reduce_partials<8>(r.part_r + r0, r.grid_r, rn, a);
    reduce_partials<10>(r.part_c + c0, r.grid_c, cn, b);
    for (int k = 0; k < kPartR; ++k) pr[k] = k < 8 ? a[k] : 0.0;
    for (int k = 0; k < kPartC; ++k) pc[k] = k < 10 ? b[k] : 0.0;
  }
  if (threadIdx.x != 0) return;
  double relk[2], gap2[2];
  for (int k = 0; k < 2; ++k) {
    const double pobj = pc[4 + k];
    const double dobj = pr[4 + k] + pc[6 + k];
    const double gap = fabs(pobj - dobj);
    st->pobj[k] = pobj;
    st->dobj[k] = dobj;
    st->relp[k] = sqrt(pr[0 + k]) / (1.0 + st->norm_q);
    st->reld[k] = sqrt(pc[0 + k]) / (1.0 + st->norm_c);
    st->relgap[k] = gap / (1.0 + fabs(pobj) + fabs(dobj));
    relk[k] = fmax(st->relp[k], fmax(st->reld[k], st->relgap[k]));
    gap2[k] = gap * gap;
  }
  if (st->init_pending) {  // KKT of the starting point: the first "last restart" data
    st->last_rp2 = pr[2];
    st->last_rd2 = pc[2];
    st->last_gap2 = gap2[0];
    st->prev_cand = INFINITY;
    st->restart_kind = 3;
    st->init_pending = 0;
    st->used_avg = 0;
    return;
  }
  st->checks += 1;
  const int use_avg_out = relk[1] < relk[0];
  st->used_avg = use_avg_out;
  const double best = use_avg_out ? relk[1] : relk[0];
  if (!isfinite(relk[0]) && !isfinite(relk[1])) {
    st->status = 4;  // PDLP_NUMERICAL
  } else if (st->terminate && best <= st->tol) {
    st->status = 1;  // PDLP_OPTIMAL
  } else if (r.rays && st->terminate && st->detect_inf &&
             inf_certificate(pr[9] + pc[11], pr[10] + pc[12], sqrt(pc[10]))) {
    // A12: y^ proves that no x satisfies the rows within the bounds
    st->status = 5;  // PDLP_PRIMAL_INFEASIBLE
    st->ray_obj = pr[9] + pc[11];
    st->ray_res = sqrt(pc[10]);
  } else if (r.rays && st->terminate && st->detect_inf &&
             inf_certificate(-pc[13], pc[14], sqrt(pr[8]))) {
    // A12: x^ is a direction of unbounded descent
    st->status = 6;  // PDLP_DUAL_INFEASIBLE
    st->ray_obj = pc[13];
    st->ray_res = sqrt(pr[8]);
  } else if (st->iters >= st->iter_limit) {
    st->status = 2;  // PDLP_ITER_LIMIT
  } else if (st->force_final) {
    st->status = 3;  // PDLP_TIME_LIMIT
  }
  st->restart_kind = 0;
  if (st->status == 0 && st->restarts_on && st->iters % st->period == 0 && st->halpern) {
    // Halpern variant: the A9 rules on the fixed-point residual of the latest step
    // against the epoch's first (prev_cand: the residual at the previous check)
    const double rr = st->h_res, r0 = st->h_r0;
    const bool do_restart = rr <= 0.2 * r0 || (rr <= 0.8 * r0 && rr > st->prev_cand) ||
                            (double)(st->iters - st->last_restart_it) >= 0.36 * (double)st->iters;
    if (!do_restart) {
      st->prev_cand = rr;
    } else {
      // A10 from the candidate's scaled distance to the previous anchor
      const double om = st->omega;
      const double ddx = sqrt(pc[8]), ddy = sqrt(pr[6]);
      if (ddx > 1e-10 && ddy > 1e-10) {
        st->omega = exp(0.5 * log(ddy / ddx) + 0.5 * log(om));
        st->inv_omega = 1.0 / st->omega;
        st->omega_f = (float)st->omega;
        st->inv_omega_f = (float)st->inv_omega;
        st->tau_d = st->eta / st->omega;
        st->sigma_d = st->eta * st->omega;
        st->tau_f = st->eta_f * st->inv_omega_f;
        st->sigma_f = st->eta_f * st->omega_f;
      }
      st->prev_cand = INFINITY;
      st->last_restart_it = st->iters;
      st->restarts += 1;
      st->restart_kind = 1;
    }
  } else if (st->status == 0 && st->restarts_on && st->iters % st->period == 0) {
    // A9: KKT restart on the scaled KKT_omega (A9b: on the normalized duality gap)
    const double om = st->omega;
    const bool ndg = st->restart_metric == 1 && r.ndg != nullptr;
    const double mc = ndg ? r.ndg->c[0].rho : kkt_omega(om, pr[2], pc[2], gap2[0]);
    const double ma = ndg ? r.ndg->c[1].rho : kkt_omega(om, pr[3], pc[3], gap2[1]);
    const int ua = ma < mc;
    const double mcand = ua ? ma : mc;
    const double mlast = ndg ? st->ndg_last : kkt_omega(om, st->last_rp2, st->last_rd2, st->last_gap2);
    const bool do_restart = mcand <= 0.2 * mlast ||
                            (mcand <= 0.8 * mlast && mcand > st->prev_cand) ||
                            (double)(st->iters - st->last_restart_it) >= 0.36 * (double)st->iters;
    if (!do_restart) {
      st->prev_cand = mcand;
    } else {
      // A10: primal weight from the scaled distances moved since the last restart
      const double ddx = sqrt(pc[8 + ua]), ddy = sqrt(pr[6 + ua]);
      if (ddx > 1e-10 && ddy > 1e-10) {
        st->omega = exp(0.5 * log(ddy / ddx) + 0.5 * log(om));
        // step scalars of the next attempt in both precisions
        st->inv_omega = 1.0 / st->omega;
        st->omega_f = (float)st->omega;
        st->inv_omega_f = (float)st->inv_omega;
        st->tau_d = st->eta / st->omega;
        st->sigma_d = st->eta * st->omega;
        st->tau_f = st->eta_f * st->inv_omega_f;
        st->sigma_f = st->eta_f * st->omega_f;
      }
      st->last_rp2 = pr[2 + ua];
      st->last_rd2 = pc[2 + ua];
      st->last_gap2 = gap2[ua];
      st->ndg_last = mcand;
      st->prev_cand = INFINITY;
      st->last_restart_it = st->iters;
      st->restarts += 1;
      st->restart_kind = ua ? 2 : 1;
    }
  }
  const long long t = st->checks - 1;
  if (t < st->tr_check_cap) {
    st->tr_restart[t] = (signed char)st->restart_kind;
    st->tr_omega[t] = st->omega;
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_kkt_apply(KktRaw r) {
  pdl_enter();
  const ESpan es = make_espan(r);
  DevState* st = r.st + es.lp;
  if (!st->check_due || st->status != 0) return;
  const int kind = st->restart_kind;
  if (kind == 0) return;
  const int cur = st->cur;
  const double pw = st->pending_w, sw = st->sum_w;
  vec2_t<T>* x = (vec2_t<T>*)r.x[cur];
  T* y = (T*)r.y[cur];
  T* sx = (T*)r.sum_x;
  T* sy = (T*)r.sum_y;
  __shared__ double inv_sh;
  if (threadIdx.x == 0) inv_sh = sw > 0.0 ? 1.0 / sw : 0.0;
  __syncthreads();
  const double isw = inv_sh;
  const long long stride = (long long)es.nblk * kBlock;
  // Halpern variant: the candidate T(z) (the current buffers) becomes the iterate and
  // the anchor
  T* hx = (T*)r.hx;
  T* hy = (T*)r.hy;
  T* hax = (T*)r.hax;
  T* hay = (T*)r.hay;
  for (long long j = es.c0 + (long long)es.bidx * kBlock + threadIdx.x; j < es.c0 + es.nc; j += stride) {
    if (hx) {
      const T xc = x[j].x;
      hx[j] = xc;
      hax[j] = xc;
    }
    if (kind == 2) {
      const double xc = (double)x[j].x;
      vec2_t<T> v;
      v.x = (T)(sw > 0.0 ? avg_of((double)sx[j] + pw * xc, sw, isw) : xc);
      v.y = (T)0;  // the step into the restart point is never read
      x[j] = v;
      r.Xl[j] = cand2(r.XG, j).y;
    } else {
      r.Xl[j] = cand2(r.XG, j).x;
    }
    if (!hx) sx[j] = (T)0;  // (the Halpern iterate lives where the sums would)
  }
  for (long long i = es.r0 + (long long)es.bidx * kBlock + threadIdx.x; i < es.r0 + es.nr; i += stride) {
    if (hy) {
      const T yc = y[i];
      hy[i] = yc;
      hay[i] = yc;
    }
    if (kind == 2) {
      const double yc = (double)y[i];
      y[i] = (T)(sw > 0.0 ? avg_of((double)sy[i] + pw * yc, sw, isw) : yc);
      r.Yl[i] = cand2(r.YG, i).y;
    } else {
      r.Yl[i] = cand2(r.YG, i).x;
    }
    if (!hy) sy[i] = (T)0;
  }
}

__global__ void k_kkt_end(KktRaw r) {
  pdl_enter();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per LP
  if (k >= r.count) return;
  DevState* st = r.st + k;
  if (!st->check_due || st->status != 0) return;
  if (st->restart_kind != 0) {
    st->sum_w = 0.0;
    st->pending_w = 0.0;
    st->pw_f = 0.0f;
    if (st->halpern) {  // a new epoch: k = 0
      st->h_k = 0;
      halpern_coeffs(st);
    }
  }
  st->restart_kind = 0;
  st->check_due = 0;
  if (r.ndg && k == 0) r.ndg->stage = 0;  // the next check's gaps start from stage 0
}

__global__ void __launch_bounds__(kBlock) k_output(KktRaw r, double* x_out, double* y_out,
                                                   double* x_cur, double* y_cur, double* x_avg,
                                                   double* y_avg) {
  const ESpan es = make_espan(r);
  const int ua = r.st[es.lp].used_avg;
  // a certificate replaces the primal (unbounded) or dual (infeasible) output
  const int status = r.st[es.lp].status;
  const bool x_ray = r.rays == 2 && status == 6, y_ray = r.rays && status == 5;
  const long long stride = (long long)es.nblk * kBlock;
  for (long long j = es.c0 + (long long)es.bidx * kBlock + threadIdx.x; j < es.c0 + es.nc; j += stride) {
    const double l = r.l[j], u = r.u[j];
    const double2 x2 = cand2(r.XG, j);
    const double xc = fmin(fmax(x2.x, l), u), xa = fmin(fmax(x2.y, l), u);
    if (x_out) x_out[j] = x_ray ? r.XR[j] : ua ? xa : xc;
    if (x_cur) x_cur[j] = xc;
    if (x_avg) x_avg[j] = xa;
  }
  for (long long i = es.r0 + (long long)es.bidx * kBlock + threadIdx.x; i < es.r0 + es.nr; i += stride) {
    const double s = r.row_kind[i] == 2 ? -1.0 : 1.0;
    const double2 y2 = cand2(r.YG, i);
    const double yc = s * y2.x, ya = s * y2.y;
    if (y_out) y_out[i] = y_ray ? s * r.YR[i] : ua ? ya : yc;
    if (y_cur) y_cur[i] = yc;
    if (y_avg) y_avg[i] = ya;
  }
}

// elementwise kernels: grid_e blocks for one LP, the A^T block map (grid_c) for a batch
inline int egrid(const KktRaw& r) { return r.tc.blk_lp ? r.grid_c : r.grid_e; }

template <int LANES, int RAYS>
cudaError_t launch_rc_mode(int which, const KktRaw& r, cudaStream_t s) {
  if (which == KK_ROWS) return launch_pdl(k_kkt_rows<LANES, RAYS>, r.grid_r, kBlock, s, r);
  return launch_pdl(k_kkt_cols<LANES, RAYS>, r.grid_c, kBlock, s, r);
}

template <int LANES>
cudaError_t launch_rc(int which, const KktRaw& r, cudaStream_t s) {
  switch (r.rays) {
    case 0: return launch_rc_mode<LANES, 0>(which, r, s);
    case 1: return launch_rc_mode<LANES, 1>(which, r, s);
    default: return launch_rc_mode<LANES, 2>(which, r, s);
  }
}

cudaError_t launch_rc_lanes(int which, int lanes, const KktRaw& r, cudaStream_t s) {
  switch (lanes) {
    case 2: return launch_rc<2>(which, r, s);
    case 4: return launch_rc<4>(which, r, s);
    case 8: return launch_rc<8>(which, r, s);
    case 16: return launch_rc<16>(which, r, s);
    case 32: return launch_rc<32>(which, r, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_kkt(int which, int lanes_r, int lanes_c, const KktRaw& r, cudaStream_t s) {
  switch (which) {
    case KK_PREP:
      if (r.fp32) return launch_pdl(k_kkt_prep<float>, egrid(r), kBlock, s, r);
      return launch_pdl(k_kkt_prep<double>, egrid(r), kBlock, s, r);
    case KK_ROWS: return launch_rc_lanes(KK_ROWS, lanes_r, r, s);
    case KK_COLS: return launch_rc_lanes(KK_COLS, lanes_c, r, s);
    case KK_FINAL:
      return launch_pdl(k_kkt_final, r.count, kBlock, s, r);
    case KK_APPLY:
      if (r.fp32) return launch_pdl(k_kkt_apply<float>, egrid(r), kBlock, s, r);
      return launch_pdl(k_kkt_apply<double>, egrid(r), kBlock, s, r);
    case KK_END:
      return launch_pdl(k_kkt_end, (r.count + kBlock - 1) / kBlock, kBlock, s, r);
    case KK_NDG:
      return launch_pdl(k_ndg_eval, r.grid_e, kBlock, s, r);
    case KK_NDG_BLOCK:
      return launch_pdl(k_ndg_block, 1, kBlock, s, r);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_output(const KktRaw& r, double* x_out, double* y_out, double* x_cur,
                          double* y_cur, double* x_avg, double* y_avg, cudaStream_t s) {
  k_output<<<egrid(r), kBlock, 0, s>>>(r, x_out, y_out, x_cur, y_cur, x_avg, y_avg);
  return cudaGetLastError();
}

}  // namespace pdlp
