// Fix-and-propagate consumer of the LP solution (section 2 of the paper):
// variable strategies Frac / RedCost / Dual / Type, LP-based randomized
// fixing, the integer-aware branching of Alg. 1, linear activity propagation
// with depth-first backtracking, and the final LP with every integer fixed,
// solved by pdlp_solve.  Host code: the paper measures this part at <= 5.5 %
// of the heuristic's time (section 4.1, time breakdown table).
//
// Readings where the paper is silent: SplitMix64 random numbers, one draw per
// branching node, u = (r >> 11) * 2^-53; the LP value is clamped to the
// current domain before its fractional part is taken; fixing goes to floor(x)
// when d > d_i, else to ceil(x); linear activity bound tightening is the only
// propagator (clique/implication propagation and repair come from code the
// paper cites but does not describe); node limit 10 |I| by default; rows are
// satisfied to 1e-6 relative (the paper's feasibility tolerance, section 4).
//
// Every floating-point operation is written in a fixed order (this file is
// compiled without FMA contraction), so integer decisions are reproducible.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "../../include/pdlp.h"

#include <string>

namespace pdlp {
extern thread_local std::string g_last_error;  // pdlp_last_error (defined with the solver)
}

namespace {

constexpr double kIntEps = 1e-6;
constexpr double kFeasTol = 1e-6;

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
};

struct Change {
  double lo, hi;
};

// at most three alternatives per branching node, kept in place (no allocation per node)
struct Alts {
  Change c[3];
  int n = 0;
  void push_back(Change x) { c[n++] = x; }
  bool empty() const { return n == 0; }
  Change back() const { return c[n - 1]; }
  void pop_back() { --n; }
};

// Alg. 1: bound changes of integer x_i with fixing value a, increasing priority
void branching(double l, double u, double a, double c, Alts& out) {
  out.n = 0;
  if (l < a && a < u) {
    if (c > 0) {
      out.push_back({a + 1, u});
      out.push_back({l, a - 1});
    } else {
      out.push_back({l, a - 1});
      out.push_back({a + 1, u});
    }
    out.push_back({a, a});
  } else if (a == l) {
    out.push_back({u, u});
    out.push_back({l, l});
  } else {
    out.push_back({l, l});
    out.push_back({u, u});
  }
}

double lp_fixing_value(double x_lp, double lo, double hi, double d) {
  const double x = std::min(std::max(x_lp, lo), hi);
  const double fl = floor(x);
  const double di = x - fl;
  return d > di ? fl : ceil(x);
}

struct Problem {
  int m, n;
  const int64_t* rp;
  const int32_t* col;
  const double* val;
  const double* b;
  const char* sense;
  const double* c;
  const double* l;
  const double* u;
  std::vector<int64_t> at_ptr;  // rows of each column, ascending
  std::vector<int32_t> at_row;
  std::vector<double> at_val;   // the matching coefficients
};

// Row activities kept up to date as bounds change: a filter only.  A row whose cached
// slack clears, with a margin, the largest range its entries had at the root is one
// whose full pass could neither find it infeasible nor tighten a bound, so the pass is
// skipped; every other row runs the full pass, which recomputes the activities exactly
// (as the oracle does) and resets the cache.  The margin (2e-9 of the row's magnitude)
// exceeds the rounding an incremental sum gathers over the 2^20 updates allowed
// between two exact recomputations.
struct RowAct {
  std::vector<double> minact, maxact;  // finite parts
  std::vector<int32_t> ninf_min, ninf_max;
  std::vector<double> range0;          // max_j |a_ij| (u_j - l_j) at the root (inf if unbounded)
  std::vector<double> mag0;            // sum_j |a_ij| 2 max(|l_j|, |u_j|), finite bounds
  std::vector<uint32_t> updates;
  static constexpr uint32_t kMaxUpdates = 1u << 20;

  // contribution of bound b (a finite value, or +-inf) to an activity
  static void add(double& act, int32_t& ninf, double a, double b, int sign) {
    if (isinf(b)) ninf += sign;
    else act += sign > 0 ? a * b : -(a * b);
  }
  // column j (entries of the column lists) moves from [olo, ohi] to [nlo, nhi]
  void change(const Problem& P, int j, double olo, double ohi, double nlo, double nhi) {
    for (int64_t q = P.at_ptr[j]; q < P.at_ptr[j + 1]; ++q) {
      const int i = P.at_row[q];
      const double a = P.at_val[q];
      const bool pos = a > 0;
      add(minact[i], ninf_min[i], a, pos ? olo : ohi, -1);
      add(minact[i], ninf_min[i], a, pos ? nlo : nhi, +1);
      add(maxact[i], ninf_max[i], a, pos ? ohi : olo, -1);
      add(maxact[i], ninf_max[i], a, pos ? nhi : nlo, +1);
      if (updates[i] < kMaxUpdates) ++updates[i];
    }
  }
  bool quiet(const Problem& P, int i) const {
    if (updates[i] >= kMaxUpdates) return false;
    const char sn = P.sense[i];
    const bool le = sn == 'L' || sn == 'E', ge = sn == 'G' || sn == 'E';
    const double bi = P.b[i];
    const double need = range0[i] + 2e-9 * (fabs(bi) + mag0[i]);
    const bool q_le = !le || ninf_min[i] >= 2 || (ninf_min[i] == 0 && bi - minact[i] >= need);
    const bool q_ge = !ge || ninf_max[i] >= 2 || (ninf_max[i] == 0 && maxact[i] - bi >= need);
    return q_le && q_ge;
  }
};

struct Domains {
  std::vector<double> lo, hi;
  std::vector<uint8_t> is_int;
  struct Entry {
    int j;
    double lo, hi;
  };
  std::vector<Entry> trail;
  const Problem* P = nullptr;  // with act: row activities follow every change
  RowAct* act = nullptr;
  void set(int j, double l, double h) {
    trail.push_back({j, lo[j], hi[j]});
    if (act) act->change(*P, j, lo[j], hi[j], l, h);
    lo[j] = l;
    hi[j] = h;
  }
  void undo(size_t mark) {
    while (trail.size() > mark) {
      const Entry e = trail.back();
      trail.pop_back();
      if (act) act->change(*P, e.j, lo[e.j], hi[e.j], e.lo, e.hi);
      lo[e.j] = e.lo;
      hi[e.j] = e.hi;
    }
  }
};

// derived bounds for column j; returns true when infeasible
bool tighten(Domains& d, int j, double new_lo, double new_hi, bool* changed) {
  const double lo = d.lo[j], hi = d.hi[j];
  double nlo, nhi;
  if (d.is_int[j]) {
    if (new_lo > -INFINITY) new_lo = ceil(new_lo - kIntEps);
    if (new_hi < INFINITY) new_hi = floor(new_hi + kIntEps);
    nlo = std::max(lo, new_lo);
    nhi = std::min(hi, new_hi);
    *changed = nlo > lo || nhi < hi;
  } else {
    nlo = new_lo > lo + 1e-7 * std::max(1.0, fabs(lo)) ? new_lo : lo;
    nhi = new_hi < hi - 1e-7 * std::max(1.0, fabs(hi)) ? new_hi : hi;
    *changed = nlo != lo || nhi != hi;
  }
  if (nlo > nhi + kIntEps) return true;
  if (*changed) d.set(j, nlo, d.is_int[j] ? nhi : std::max(nhi, nlo));
  return false;
}

// linear activity bound tightening to a fixpoint, FIFO over rows; false if infeasible
bool propagate(const Problem& P, Domains& d, const int32_t* rows, int64_t nrows,
               std::vector<uint8_t>& inq, std::vector<int32_t>& queue) {
  queue.clear();
  for (int64_t k = 0; k < nrows; ++k) {
    const int i = rows[k];
    if (!inq[i]) {
      inq[i] = 1;
      queue.push_back(i);
    }
  }
  bool ok = true;
  size_t head = 0;
  while (head < queue.size()) {
    const int i = queue[head++];
    inq[i] = 0;
    if (!ok) continue;  // drain the queue flags
    if (d.act && d.act->quiet(P, i)) continue;
    const int64_t s = P.rp[i], e = P.rp[i + 1];
    const double bi = P.b[i];
    const char sn = P.sense[i];
    const bool le = sn == 'L' || sn == 'E', ge = sn == 'G' || sn == 'E';
    double minact = 0.0, maxact = 0.0;
    double maxrange = 0.0, mag = 0.0;  // largest |a_j| (hi_j - lo_j); sum of |a_j| |bounds|
    int ninf_min = 0, ninf_max = 0;
    for (int64_t p = s; p < e; ++p) {
      const double a = P.val[p];
      const int j = P.col[p];
      const double lo = d.lo[j], hi = d.hi[j];
      if (a > 0) {
        if (lo == -INFINITY) ++ninf_min; else minact += a * lo;
        if (hi == INFINITY) ++ninf_max; else maxact += a * hi;
      } else {
        if (hi == INFINITY) ++ninf_min; else minact += a * hi;
        if (lo == -INFINITY) ++ninf_max; else maxact += a * lo;
      }
      maxrange = std::max(maxrange, fabs(a) * (hi - lo));
      mag += fabs(a) * ((lo > -INFINITY ? fabs(lo) : 0.0) + (hi < INFINITY ? fabs(hi) : 0.0));
    }
    if (d.act) {  // the exact activities replace the cached ones
      d.act->minact[i] = minact;
      d.act->maxact[i] = maxact;
      d.act->ninf_min[i] = ninf_min;
      d.act->ninf_max[i] = ninf_max;
      d.act->updates[i] = 0;
    }
    const double tol = kFeasTol * std::max(1.0, fabs(bi));
    if ((le && ninf_min == 0 && minact > bi + tol) || (ge && ninf_max == 0 && maxact < bi - tol)) {
      ok = false;
      continue;
    }
    // No entry can be tightened when the row's slack covers every entry's whole range
    // (with a margin far above the rounding of the activities), or when two or more
    // entries are unbounded on the side that would derive a bound: skip the pass.
    const double margin = 1e-9 * (fabs(bi) + mag);
    const bool quiet_le = !le || ninf_min >= 2 || (ninf_min == 0 && bi - minact >= maxrange + margin);
    const bool quiet_ge = !ge || ninf_max >= 2 || (ninf_max == 0 && maxact - bi >= maxrange + margin);
    if (quiet_le && quiet_ge) continue;
    for (int64_t p = s; p < e && ok; ++p) {
      const double a = P.val[p];
      const int j = P.col[p];
      const double lo = d.lo[j], hi = d.hi[j];
      double new_lo = -INFINITY, new_hi = INFINITY;
      if (le) {
        const double own = a > 0 ? a * lo : a * hi;
        const bool own_inf = a > 0 ? lo == -INFINITY : hi == INFINITY;
        if (ninf_min == 0 || (ninf_min == 1 && own_inf)) {
          const double rest = minact - (own_inf ? 0.0 : own);
          const double bound = (bi - rest) / a;
          if (a > 0) new_hi = bound; else new_lo = bound;
        }
      }
      if (ge) {
        const double own = a > 0 ? a * hi : a * lo;
        const bool own_inf = a > 0 ? hi == INFINITY : lo == -INFINITY;
        if (ninf_max == 0 || (ninf_max == 1 && own_inf)) {
          const double rest = maxact - (own_inf ? 0.0 : own);
          const double bound = (bi - rest) / a;
          if (a > 0) new_lo = std::max(new_lo, bound); else new_hi = std::min(new_hi, bound);
        }
      }
      bool changed = false;
      if (tighten(d, j, new_lo, new_hi, &changed)) {
        ok = false;
        break;
      }
      if (changed) {
        for (int64_t q = P.at_ptr[j]; q < P.at_ptr[j + 1]; ++q) {
          const int r = P.at_row[q];
          if (r != i && !inq[r]) {
            inq[r] = 1;
            queue.push_back(r);
          }
        }
      }
    }
  }
  for (size_t k = head; k < queue.size(); ++k) inq[queue[k]] = 0;
  return ok;
}

static double fractionality(double v) { return std::min(v - floor(v), ceil(v) - v); }

// DUAL: rows by descending |y| (stable); each row's integers not yet seen by
// descending |lambda| -- with `frac`, then by ascending fractionality -- in storage
// order otherwise; the integers of no row last, by index (with `frac`: by ascending
// fractionality, then index).
static void dual_order(const Problem& P, const std::vector<double>& lam, const double* y_lp,
                       const uint8_t* is_int, const std::vector<double>* frac,
                       std::vector<int>& order) {
  std::vector<int> rows(P.m);
  for (int i = 0; i < P.m; ++i) rows[i] = i;
  std::stable_sort(rows.begin(), rows.end(),
                   [&](int a, int b) { return fabs(y_lp[a]) > fabs(y_lp[b]); });
  std::vector<uint8_t> seen(P.n, 0);
  std::vector<int> cols;
  for (int i : rows) {
    cols.clear();
    for (int64_t p = P.rp[i]; p < P.rp[i + 1]; ++p) {
      const int j = P.col[p];
      if (is_int[j] && !seen[j]) cols.push_back(j);
    }
    std::stable_sort(cols.begin(), cols.end(), [&](int a, int b) {
      const double la = fabs(lam[a]), lb = fabs(lam[b]);
      if (la != lb) return la > lb;
      return frac ? (*frac)[a] < (*frac)[b] : false;
    });
    for (int j : cols)
      if (!seen[j]) {
        seen[j] = 1;
        order.push_back(j);
      }
  }
  std::vector<int> rest;
  for (int j = 0; j < P.n; ++j)
    if (is_int[j] && !seen[j]) rest.push_back(j);
  if (frac)
    std::stable_sort(rest.begin(), rest.end(), [&](int a, int b) { return (*frac)[a] < (*frac)[b]; });
  order.insert(order.end(), rest.begin(), rest.end());
}

void variable_order(const Problem& P, int strategy, const double* x_lp, const double* y_lp,
                    const uint8_t* is_int, std::vector<int>& order) {
  std::vector<int> ints;
  for (int j = 0; j < P.n; ++j)
    if (is_int[j]) ints.push_back(j);
  order.clear();
  std::vector<double> frac(P.n);
  for (int j = 0; j < P.n; ++j) frac[j] = fractionality(x_lp[j]);
  if (strategy == FP_FRAC) {
    order = ints;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return frac[a] < frac[b]; });
    return;
  }
  if (strategy == FP_TYPE) {
    for (int j : ints)
      if (P.l[j] == 0.0 && P.u[j] == 1.0) order.push_back(j);
    for (int j : ints)
      if (!(P.l[j] == 0.0 && P.u[j] == 1.0)) order.push_back(j);
    return;
  }
  // reduced costs lambda = c - A^T y, accumulated row by row
  std::vector<double> lam(P.c, P.c + P.n);
  for (int i = 0; i < P.m; ++i)
    for (int64_t p = P.rp[i]; p < P.rp[i + 1]; ++p) lam[P.col[p]] -= P.val[p] * y_lp[i];
  switch (strategy) {
    case FP_REDCOST:
      order = ints;
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int b) { return fabs(lam[a]) > fabs(lam[b]); });
      return;
    case FP_DUAL:
      dual_order(P, lam, y_lp, is_int, nullptr, order);
      return;
    case FP_FRAC_DUAL: {  // fractionality, ties by position in the DUAL order
      std::vector<int> dual;
      dual_order(P, lam, y_lp, is_int, nullptr, dual);
      std::vector<int> rank(P.n, 0);
      for (size_t k = 0; k < dual.size(); ++k) rank[dual[k]] = (int)k;
      order = ints;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (frac[a] != frac[b]) return frac[a] < frac[b];
        return rank[a] < rank[b];
      });
      return;
    }
    case FP_FRAC_REDCOST:  // fractionality, ties by descending |lambda|, then index
      order = ints;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (frac[a] != frac[b]) return frac[a] < frac[b];
        return fabs(lam[a]) > fabs(lam[b]);
      });
      return;
    case FP_DUAL_FRAC:
      dual_order(P, lam, y_lp, is_int, &frac, order);
      return;
    default:  // FP_REDCOST_FRAC: descending |lambda|, ties by fractionality, then index
      order = ints;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double la = fabs(lam[a]), lb = fabs(lam[b]);
        if (la != lb) return la > lb;
        return frac[a] < frac[b];
      });
      return;
  }
}

// Largest row violation of x, each scaled by max(1, |b_i|) (the paper's
// relative feasibility tolerance, section 4, read per row).
double max_row_violation(const Problem& P, const double* x) {
  double worst = 0.0;
  for (int i = 0; i < P.m; ++i) {
    double act = 0.0;
    for (int64_t p = P.rp[i]; p < P.rp[i + 1]; ++p) act += P.val[p] * x[P.col[p]];
    const double bi = P.b[i];
    double v = 0.0;
    if (P.sense[i] == 'L') v = act - bi;
    else if (P.sense[i] == 'G') v = bi - act;
    else v = fabs(act - bi);
    worst = std::max(worst, v / std::max(1.0, fabs(bi)));
  }
  return worst;
}

int fp_fail(fp_result* r, int status) {
  r->status = status;
  r->obj = NAN;
  return PDLP_OK;
}

// a rejected argument: PDLP_ERR_INVALID_INPUT with its reason for pdlp_last_error
int bad_input(const char* why) {
  pdlp::g_last_error = why;
  return PDLP_ERR_INVALID_INPUT;
}

}  // namespace

extern "C" int fp_default_params(fp_params* p) {
  if (!p) return PDLP_ERR_INVALID_INPUT;
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(fp_params);
  p->var_strategy = FP_TYPE;
  p->seed = 1;
  p->node_limit = 0;
  p->final_lp = 1;
  p->final_lp_tol = 1e-8;
  return PDLP_OK;
}

extern "C" int fp_run(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const double* x_lp, const double* y_lp,
                      const uint8_t* is_int, const fp_params* prm, double* x_out, fp_result* r) {
  fp_params dflt;
  if (!prm) {
    fp_default_params(&dflt);
    prm = &dflt;
  }
  if (!A || !r || !x_out || !is_int || !x_lp || !c || !l || !u || (A->m > 0 && (!b || !sense)))
    return bad_input("fp_run: NULL problem, vector, result or output argument");
  if (prm->struct_size != sizeof(fp_params))
    return bad_input("fp_params.struct_size mismatch (use fp_default_params)");
  if (A->m < 0 || A->n < 1 || A->nnz < 0) return bad_input("fp_run: need m >= 0, n >= 1, nnz >= 0");
  if (prm->var_strategy < FP_FRAC || prm->var_strategy > FP_REDCOST_FRAC)
    return bad_input("fp_run: unknown var_strategy");
  if (prm->var_strategy != FP_FRAC && prm->var_strategy != FP_TYPE && !y_lp && A->m > 0)
    return bad_input("fp_run: FP_REDCOST, FP_DUAL and the hybrid strategies need y_lp");
  memset(r, 0, sizeof(*r));
  const auto t0 = std::chrono::steady_clock::now();
  Problem P{A->m, A->n, A->row_ptr, A->col, A->val, b, sense, c, l, u, {}, {}, {}};
  // column lists, rows ascending
  P.at_ptr.assign(P.n + 1, 0);
  for (int64_t p = 0; p < A->nnz; ++p) {
    if (A->col[p] < 0 || A->col[p] >= P.n) return bad_input("fp_run: column index out of range");
    ++P.at_ptr[A->col[p] + 1];
  }
  for (int j = 0; j < P.n; ++j) P.at_ptr[j + 1] += P.at_ptr[j];
  P.at_row.resize(A->nnz);
  P.at_val.resize(A->nnz);
  {
    std::vector<int64_t> cur(P.at_ptr.begin(), P.at_ptr.end() - 1);
    for (int i = 0; i < P.m; ++i)
      for (int64_t p = P.rp[i]; p < P.rp[i + 1]; ++p) {
        const int64_t q = cur[P.col[p]]++;
        P.at_row[q] = i;
        P.at_val[q] = P.val[p];
      }
  }
  Domains d;
  d.lo.assign(l, l + P.n);
  d.hi.assign(u, u + P.n);
  d.is_int.assign(is_int, is_int + P.n);
  int64_t n_int = 0;
  for (int j = 0; j < P.n; ++j) {
    if (!is_int[j]) continue;
    ++n_int;
    if (isfinite(d.lo[j])) d.lo[j] = ceil(d.lo[j] - kIntEps);
    if (isfinite(d.hi[j])) d.hi[j] = floor(d.hi[j] + kIntEps);
  }
  const int64_t limit = prm->node_limit > 0 ? prm->node_limit : 10 * n_int;
  // row activities of the root domains, then kept up to date by every bound change
  RowAct act;
  act.minact.assign(P.m, 0.0);
  act.maxact.assign(P.m, 0.0);
  act.ninf_min.assign(P.m, 0);
  act.ninf_max.assign(P.m, 0);
  act.range0.assign(P.m, 0.0);
  act.mag0.assign(P.m, 0.0);
  act.updates.assign(P.m, 0);
  for (int i = 0; i < P.m; ++i)
    for (int64_t p = P.rp[i]; p < P.rp[i + 1]; ++p) {
      const double a = P.val[p];
      const int j = P.col[p];
      const double lo = d.lo[j], hi = d.hi[j];
      RowAct::add(act.minact[i], act.ninf_min[i], a, a > 0 ? lo : hi, +1);
      RowAct::add(act.maxact[i], act.ninf_max[i], a, a > 0 ? hi : lo, +1);
      act.range0[i] = std::max(act.range0[i], fabs(a) * (hi - lo));
      act.mag0[i] += fabs(a) * 2.0 *
                     std::max(isfinite(lo) ? fabs(lo) : 0.0, isfinite(hi) ? fabs(hi) : 0.0);
    }
  d.P = &P;
  d.act = &act;
  std::vector<uint8_t> inq(P.m, 0);
  std::vector<int32_t> queue, all_rows(P.m);
  for (int i = 0; i < P.m; ++i) all_rows[i] = i;
  if (!propagate(P, d, all_rows.data(), P.m, inq, queue)) return fp_fail(r, FP_INFEASIBLE);
  std::vector<int> order;
  variable_order(P, prm->var_strategy, x_lp, y_lp, is_int, order);
  SplitMix64 rng{prm->seed};
  struct Frame {
    size_t mark;
    int var;
    size_t pos;  // position of var in the order
    Alts alts;
  };
  std::vector<Frame> frames;
  int status = 0;
  while (true) {
    // the first integer of the order that is not fixed yet.  Every integer before the
    // top frame's position was fixed when that frame was made, and the search below it
    // only undoes to that state or narrows domains, so the scan starts there (a scan
    // from the front made the search quadratic in the number of integers)
    int j = -1;
    size_t pos = frames.empty() ? 0 : frames.back().pos;
    for (; pos < order.size(); ++pos) {
      const int v = order[pos];
      if (d.hi[v] - d.lo[v] > 0.5) {
        j = v;
        break;
      }
    }
    if (j < 0) {
      status = FP_FEASIBLE;
      break;
    }
    if (r->nodes >= limit) {
      status = FP_NODE_LIMIT;
      break;
    }
    ++r->nodes;
    const double a = lp_fixing_value(x_lp[j], d.lo[j], d.hi[j], rng.uniform());
    frames.push_back({d.trail.size(), j, pos, {}});
    branching(d.lo[j], d.hi[j], a, c[j], frames.back().alts);
    bool descended = false;
    while (!descended) {
      Frame& f = frames.back();
      d.undo(f.mark);
      if (f.alts.empty()) {
        frames.pop_back();
        ++r->backtracks;
        if (frames.empty()) break;
        continue;
      }
      const Change ch = f.alts.back();
      f.alts.pop_back();
      d.set(f.var, ch.lo, ch.hi);
      if (propagate(P, d, P.at_row.data() + P.at_ptr[f.var], P.at_ptr[f.var + 1] - P.at_ptr[f.var],
                    inq, queue))
        descended = true;
    }
    if (!descended) {
      status = FP_INFEASIBLE;
      break;
    }
  }
  r->search_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int j = 0; j < P.n; ++j) x_out[j] = is_int[j] ? d.lo[j] : NAN;
  if (status != FP_FEASIBLE) return fp_fail(r, status);
  if (!prm->final_lp) {
    r->status = FP_NO_FINAL_LP;
    r->obj = NAN;
    return PDLP_OK;
  }
  // final LP: every integer fixed at its value, continuous columns keep their bounds
  std::vector<double> fl(P.n), fu(P.n), xf(P.n), yf(std::max(P.m, 1));
  for (int j = 0; j < P.n; ++j) {
    fl[j] = is_int[j] ? d.lo[j] : l[j];
    fu[j] = is_int[j] ? d.lo[j] : u[j];
  }
  // The final point counts as feasible when every row holds to kFeasTol max(1, |b_i|).
  // A first-order solution at final_lp_tol may miss a row by a little: then that
  // point is polished (the same PDHG on the objective-free problem from it).
  pdlp_params pp;
  pdlp_default_params(&pp);
  pp.tol = prm->final_lp_tol;
  pdlp_result lr;
  const auto t1 = std::chrono::steady_clock::now();
  int rc = pdlp_solve(A, b, sense, c, fl.data(), fu.data(), &pp, nullptr, nullptr, xf.data(),
                      yf.data(), &lr, nullptr);
  if (rc != PDLP_OK) return rc;
  long long lp_iters = lr.iters;
  for (int j = 0; j < P.n; ++j) x_out[j] = is_int[j] ? d.lo[j] : xf[j];
  double viol = max_row_violation(P, x_out);
  if (lr.status == PDLP_OPTIMAL && viol > kFeasTol) {
    const std::vector<double> x0(xf);
    rc = pdlp_polish_primal(A, b, sense, fl.data(), fu.data(), &pp, x0.data(), xf.data(),
                            yf.data(), &lr);
    if (rc != PDLP_OK) return rc;
    lp_iters += lr.iters;
    for (int j = 0; j < P.n; ++j) x_out[j] = is_int[j] ? d.lo[j] : xf[j];
    viol = max_row_violation(P, x_out);
  }
  r->lp_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
  r->final_lp_iters = lp_iters;
  r->final_rel_primal = lr.rel_primal_res;
  if (lr.status != PDLP_OPTIMAL || viol > kFeasTol) return fp_fail(r, FP_INFEASIBLE);
  double obj = 0.0;
  for (int j = 0; j < P.n; ++j) obj += c[j] * x_out[j];
  r->status = FP_FEASIBLE;
  r->obj = obj;
  return PDLP_OK;
}

extern "C" int fp_run_refs(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                           const double* l, const double* u, const double* const* x_refs,
                           int nrefs, const double* y_lp, const uint8_t* is_int,
                           const fp_params* prm, double* x_out, fp_result* r, int* chosen) {
  if (!A || !x_refs || nrefs < 1 || !x_out || !r || !chosen || A->n < 1)
    return bad_input("fp_run_refs: need A, nrefs >= 1 reference points, x_out, r and chosen");
  for (int k = 0; k < nrefs; ++k)
    if (!x_refs[k]) return bad_input("fp_run_refs: NULL reference point");
  std::vector<double> x((size_t)A->n);
  fp_result cur;
  bool have = false;
  *chosen = -1;
  for (int k = 0; k < nrefs; ++k) {
    const int rc = fp_run(A, b, sense, c, l, u, x_refs[k], y_lp, is_int, prm, x.data(), &cur);
    if (rc != PDLP_OK) return rc;
    const bool better = cur.status == FP_FEASIBLE && (!have || cur.obj < r->obj);
    if (better || (!have && k == nrefs - 1)) {
      *r = cur;
      std::copy(x.begin(), x.end(), x_out);
    }
    if (better) {
      have = true;
      *chosen = k;
    }
  }
  return PDLP_OK;
}
