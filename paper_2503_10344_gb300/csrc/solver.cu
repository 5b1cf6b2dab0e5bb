// Host driver of one PDLP solve and the C ABI of include/pdlp.h.
//
// Flow of pdlp_solve_device (all device work in stream order on the caller's
// stream):
//   1. carve the workspace; validate the inputs on the device (error bits);
//   2. canonical form (A0), transpose (A1), value-format check, Ruiz +
//      Pock-Chambolle scaling (A2), iteration-space matrix and vectors, the
//      scalars of A3 (one small read-back);
//   3. the KKT block once in "initial" mode: the KKT of the start point
//      becomes the first restart reference;
//   4. a CUDA graph holding `check_period` step attempts (primal + dual
//      kernels each) followed by the KKT block is launched repeatedly; after
//      each launch four bytes of state are copied to pinned host memory and
//      the host reads them one launch behind, so the GPU never waits for the
//      host.  Kernels launched after termination return at once.
//   5. outputs in the caller's convention, result struct.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <functional>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/pdlp.h"
#include "setup.h"

namespace pdlp {

thread_local std::string g_last_error;
thread_local long long g_launches = 0;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(x)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      return fail(PDLP_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));        \
  } while (0)

// ---------------------------------------------------------------- workspace
struct Arena {
  char* base;
  size_t off;
  void* take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

// Step-rule factors 1 - (k+1)^-0.3 and 1 + (k+1)^-0.6 of attempts k = 1..kFacN,
// computed once per process with the C library pow (static storage, no heap).
constexpr int kFacN = 32768;
struct FacTable {
  double dec[kFacN], inc[kFacN];
  float dec_f[kFacN], inc_f[kFacN];
};
static FacTable g_fac;
static std::once_flag g_fac_once;
static const FacTable& fac_table() {
  std::call_once(g_fac_once, [] {
    for (int i = 0; i < kFacN; ++i) {
      const double k1 = (double)(i + 1) + 1.0;
      g_fac.dec[i] = 1.0 - std::pow(k1, -0.3);
      g_fac.inc[i] = 1.0 + std::pow(k1, -0.6);
      g_fac.dec_f[i] = (float)g_fac.dec[i];
      g_fac.inc_f[i] = (float)g_fac.inc[i];
    }
  });
  return g_fac;
}

struct Bufs {
  FacTable* fac;
  int *a_ptr, *a_col, *t_ptr, *t_col;
  double *a_val64, *t_val64;
  void *a_valit, *t_valit;
  double *q64, *dr, *dc, *Xl, *Yl, *stat_r, *stat_c, *inv_dr, *inv_dc;
  double2 *XG, *YG;
  double *XR, *YR;
  unsigned char *row_kind, *bflags;
  void *c_it, *l_it, *u_it, *q_it, *tw, *sw, *x[2], *y[2], *sum_x, *sum_y;
  double *part_p, *part_d, *part_r, *part_c, *part_setup, *scalars;
  int *a_long, *t_long, *tmp, *flags2;
  int *ord_t, *ord_a;  // columns / rows longest first (the shared-memory one-block kernel)
  DevState* st;
  // staged tile kernels (float32 iterates): items over A (dual step) and A^T (primal)
  TileItem *ti_a, *ti_t;
  float2 *tpart_a, *tpart_t, *trow_a, *trow_t, *tlong_a, *tlong_t;
  int *tick_a, *tick_t, *tlp_a, *tlp_t;  // tickets; [item0[0..count], lng0[0..count]]
  size_t tcap_a, tcap_t;
  double2 *ndg_gx, *ndg_gy;  // normalized-duality-gap restarts (NULL off)
  NdgState* ndg;
  double* ndg_part;
};

constexpr int kMaxLongBlocks = 1024;
constexpr int kAttemptsPerBody = 8;  // step attempts per iteration of the graph's while loop

static int max_blocks() { return device_sm_count() * 8; }

// bytes of one iterate element and one iteration-matrix value for a precision request
static void elem_sizes(int precision, size_t* it_bytes, size_t* val_bytes) {
  if (precision == PDLP_FP64) {
    *it_bytes = 8;
    *val_bytes = 8;
  } else {
    *it_bytes = 4;
    *val_bytes = 4;  // bound: bf16 (2) / pattern (0) fit, FP32 fallback needs 4
  }
}

static size_t carve(Arena& ar, Bufs& b, int m, int n, long long nnz, int precision,
                    bool ndg = false) {
  size_t eb, vb;
  elem_sizes(precision, &eb, &vb);
  const size_t G = (size_t)max_blocks() + kMaxLongBlocks;
  const size_t M = (size_t)m, N = (size_t)n, Z = (size_t)nnz;
  b.fac = (FacTable*)ar.take(sizeof(FacTable));
  b.a_ptr = (int*)ar.take(4 * (M + 1));
  b.t_ptr = (int*)ar.take(4 * (N + 1));
  b.a_col = (int*)ar.take(4 * Z);
  b.t_col = (int*)ar.take(4 * Z);
  b.a_val64 = (double*)ar.take(8 * Z);
  b.t_val64 = (double*)ar.take(8 * Z);
  b.a_valit = ar.take(vb * Z);
  b.t_valit = ar.take(vb * Z);
  b.q64 = (double*)ar.take(8 * M);
  b.dr = (double*)ar.take(8 * M);
  b.dc = (double*)ar.take(8 * N);
  b.XG = (double2*)ar.take(16 * N);
  b.XR = (double*)ar.take(8 * N);
  b.Xl = (double*)ar.take(8 * N);
  b.YG = (double2*)ar.take(16 * M);
  b.YR = (double*)ar.take(8 * M);
  b.Yl = (double*)ar.take(8 * M);
  b.stat_r = (double*)ar.take(8 * M);
  b.stat_c = (double*)ar.take(8 * N);
  b.row_kind = (unsigned char*)ar.take(M);
  b.inv_dr = (double*)ar.take(8 * M);
  b.inv_dc = (double*)ar.take(8 * N);
  b.bflags = (unsigned char*)ar.take(N);
  b.ord_t = (int*)ar.take(4 * N);
  b.ord_a = (int*)ar.take(4 * M);
  b.c_it = ar.take(eb * N);
  b.l_it = ar.take(eb * N);
  b.u_it = ar.take(eb * N);
  b.tw = ar.take(eb * N);
  b.q_it = ar.take(eb * M);
  b.sw = ar.take(eb * M);
  for (int k = 0; k < 2; ++k) {
    b.x[k] = ar.take(2 * eb * N);  // (x_j, dx_j) pairs
    b.y[k] = ar.take(eb * M);
  }
  b.sum_x = ar.take(eb * N);
  b.sum_y = ar.take(eb * M);
  b.part_p = (double*)ar.take(8 * G);
  b.part_d = (double*)ar.take(8 * 2 * G);
  b.part_r = (double*)ar.take(8 * kPartR * G);
  b.part_c = (double*)ar.take(8 * kPartC * G);
  b.part_setup = (double*)ar.take(8 * setup_part_doubles(m, n));
  b.scalars = (double*)ar.take(8 * 8);
  b.a_long = (int*)ar.take(4 * (M + 1));
  b.t_long = (int*)ar.take(4 * (N + 1));
  const size_t tmp_ints = std::max(transpose_tmp_ints(m, n, nnz),
                                   2 * (std::max(M, N) + 1) + scan_tmp_ints((long long)std::max(M, N) + 1));
  b.flags2 = (int*)ar.take(16);
  b.st = (DevState*)ar.take(sizeof(DevState));
  b.tcap_a = b.tcap_t = 0;
  size_t tile_tmp = 0;
  if (precision != PDLP_FP64) {
    // both tile forms fit: block tiles keep one partial per warp and slot, warp tiles one
    const TileShape s1 = tile_shape(1), s2 = tile_shape(2);
    b.tcap_a = std::max(tile_item_cap(s1, m, nnz, 1), tile_item_cap(s2, m, nnz, 1));
    b.tcap_t = std::max(tile_item_cap(s1, n, nnz, 1), tile_item_cap(s2, n, nnz, 1));
    const size_t pa = std::max(kWarps * tile_item_cap(s1, m, nnz, 1), tile_item_cap(s2, m, nnz, 1));
    const size_t pt = std::max(kWarps * tile_item_cap(s1, n, nnz, 1), tile_item_cap(s2, n, nnz, 1));
    b.ti_a = (TileItem*)ar.take(sizeof(TileItem) * b.tcap_a);
    b.ti_t = (TileItem*)ar.take(sizeof(TileItem) * b.tcap_t);
    b.tpart_a = (float2*)ar.take(8 * pa);
    b.tpart_t = (float2*)ar.take(8 * pt);
    for (float2** v : {&b.trow_a, &b.tlong_a}) *v = (float2*)ar.take(8 * b.tcap_a);
    for (float2** v : {&b.trow_t, &b.tlong_t}) *v = (float2*)ar.take(8 * b.tcap_t);
    b.tick_a = (int*)ar.take(4 * b.tcap_a);
    b.tick_t = (int*)ar.take(4 * b.tcap_t);
    b.tlp_a = (int*)ar.take(4 * 4);
    b.tlp_t = (int*)ar.take(4 * 4);
    tile_tmp = tile_tmp_ints(std::max(m, n));
  }
  b.tmp = (int*)ar.take(4 * std::max(tmp_ints, tile_tmp));
  // normalized-duality-gap restarts: gradients of both candidates, bisection state, partials
  b.ndg_gx = ndg ? (double2*)ar.take(16 * N) : nullptr;
  b.ndg_gy = ndg ? (double2*)ar.take(16 * M) : nullptr;
  b.ndg = ndg ? (NdgState*)ar.take(sizeof(NdgState)) : nullptr;
  b.ndg_part = ndg ? (double*)ar.take(8 * 4 * G) : nullptr;
  return ar.off + 256;
}

// Lanes per row: the smallest power of two giving each lane at most `per_lane`
// entries of an average row, in [2, 32].  Fewer lanes put more rows in a warp
// (fewer shuffle levels, more rows per epilogue instruction); on GB300 float64
// kernels pay ~16 pipe cycles per warp instruction, so they use fewer lanes.
static int auto_lanes(double avg_len, double per_lane) {
  int l = 2;
  while (l < 32 && l * per_lane < avg_len) l <<= 1;
  return l;
}

// Lanes per row of a float32 step kernel: one lane per row (every thread sums and
// finishes whole rows: no idle lanes in the epilogue, consecutive rows on consecutive
// lanes) when an average row has at most kOneLaneAvg entries and the two-launch kernels
// run (`one_ok`), else auto_lanes.  Measured on GB300 with float32 iterates: the energy
// system (2.10M x 2.45M, 3.75 / 3.2 entries per row of A / A^T) 96.8 -> 75.6 us per
// attempt; the primal kernel of the 256 covering sub-LPs (6.5 entries per column)
// 527 -> 449 us, of the 50k x 200k covering LP 20.7 -> 19.9 us per attempt; over the
// covering rows (26 entries) one lane per row is 1.4-4x slower.
constexpr double kOneLaneAvg = 8.0;
static int step_lanes(double avg_len, double per_lane, bool one_ok) {
  return one_ok && avg_len <= kOneLaneAvg ? 1 : auto_lanes(avg_len, per_lane);
}

// Rows longer than this go to the long-row blocks (one block per row).  With one lane
// per row a thread walks its rows' entries one after another, so the cut-off is low.
static int long_thresh(int step_lanes, int kkt_lanes) {
  return step_lanes == 1 ? 64 : std::max(1024, 128 * std::max(step_lanes, kkt_lanes));
}

static bool valid_lanes(int l) { return l == 2 || l == 4 || l == 8 || l == 16 || l == 32; }
// the two-launch step kernels also take one lane per row (the persistent kernel and the
// KKT passes do not)
static bool valid_step_lanes(int l) { return l == 1 || valid_lanes(l); }

// Grid of a staged tile kernel over `items` work items with at most `resident`
// blocks at once: every block gets the same number of items, give or take one
// (ceil(items / blocks) rounds for all), in one wave.
static int tile_grid(int items, int resident) {
  if (items <= 0) return 1;
  const int rounds = (items + resident - 1) / resident;
  return (items + rounds - 1) / rounds;
}

static cudaError_t tile_resident_mode(Mode mode, int form, int* bp, int* bd) {
  switch (mode) {
    case MODE_FP32: return tile_resident_fp32(form, bp, bd);
    case MODE_BF16: return tile_resident_bf16(form, bp, bd);
    case MODE_PAT: return tile_resident_pat(form, bp, bd);
    default: return cudaErrorInvalidValue;
  }
}

// Launch shape of the tile kernels of a form over `items` work items, with `resident`
// blocks at most at once: grid (blocks) and workers (blocks, or warps for warp tiles).
static void tile_launch(int form, int items, int resident, int* grid, int* workers) {
  if (form == 2) {
    const int w = tile_grid(items, kWarps * resident);
    *grid = (w + kWarps - 1) / kWarps;
    *workers = kWarps * *grid;
  } else {
    *grid = *workers = tile_grid(items, resident);
  }
}

// ---------------------------------------------------------------- solver
struct Solve {
  int m, n;
  long long nnz;
  Mode mode;
  int lanes_a, lanes_t;    // step kernels
  int lanes_ka, lanes_kt;  // KKT passes
  IterRaw ir;
  KktRaw kr;
  cudaStream_t s;
  int persist_grid;  // > 0: one persistent kernel per check period (one LP)
  // while capturing a graph: a second stream and two events that let the KKT
  // passes over A and A^T run side by side (the first waits on memory, the second
  // on the float64 pipe); null outside a capture, where they run one after the other
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  cudaError_t persist(int max_attempts) {
    ++g_launches;
    int g = 0;
    switch (mode) {
      case MODE_FP64: return launch_persist_fp64(lanes_a, lanes_t, ir, max_attempts, persist_grid, &g, s);
      case MODE_FP32: return launch_persist_fp32(lanes_a, lanes_t, ir, max_attempts, persist_grid, &g, s);
      case MODE_BF16: return launch_persist_bf16(lanes_a, lanes_t, ir, max_attempts, persist_grid, &g, s);
      default: return launch_persist_pat(lanes_a, lanes_t, ir, max_attempts, persist_grid, &g, s);
    }
  }
  // the step attempts of one check period: one persistent launch, or two
  // launches per attempt
  cudaError_t period_steps(int period) {
    if (persist_grid > 0) return persist(4 * period);
    cudaError_t e = cudaSuccess;
    for (int a = 0; a < period && e == cudaSuccess; ++a) {
      e = iter(IK_PRIMAL);
      if (e == cudaSuccess) e = iter(IK_DUAL);
    }
    return e;
  }

  cudaError_t iter(int which) {
    g_launches += which == IK_DUAL ? 2 : 1;  // the dual step is followed by the decision
    const int lanes = which == IK_PRIMAL ? lanes_t : lanes_a;
    if (ir.hx) {  // the Halpern variant
      switch (mode) {
        case MODE_FP64: return launch_iter_fp64_h(which, lanes, ir, s);
        case MODE_FP32: return launch_iter_fp32_h(which, lanes, ir, s);
        case MODE_BF16: return launch_iter_bf16_h(which, lanes, ir, s);
        default: return launch_iter_pat_h(which, lanes, ir, s);
      }
    }
    switch (mode) {
      case MODE_FP64: return launch_iter_fp64(which, lanes, ir, s);
      case MODE_FP32: return launch_iter_fp32(which, lanes, ir, s);
      case MODE_BF16: return launch_iter_bf16(which, lanes, ir, s);
      default: return launch_iter_pat(which, lanes, ir, s);
    }
  }
  // normalized-duality-gap restarts: the stages of both candidates' gaps, after the
  // passes (which write the gradients) and before the restart decision
  cudaError_t ndg_stages() {
    if (kr.ndg == nullptr) return cudaSuccess;
    if ((long long)kr.m + kr.n <= kNdgOneBlock) {  // a small LP: every stage in one block
      ++g_launches;
      return launch_kkt(KK_NDG_BLOCK, lanes_ka, lanes_kt, kr, s);
    }
    g_launches += kNdgStages;
    for (int k = 0; k < kNdgStages; ++k) {
      const cudaError_t e = launch_kkt(KK_NDG, lanes_ka, lanes_kt, kr, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t kkt_block() {
    cudaError_t e;
    if (s2 == nullptr) {
      for (int k : {KK_PREP, KK_ROWS, KK_COLS, KK_FINAL, KK_APPLY, KK_END}) {
        if (k == KK_FINAL && (e = ndg_stages()) != cudaSuccess) return e;
        ++g_launches;
        if ((e = launch_kkt(k, lanes_ka, lanes_kt, kr, s)) != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    g_launches += 6;
    if ((e = launch_kkt(KK_PREP, lanes_ka, lanes_kt, kr, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s2, ev_fork, 0)) != cudaSuccess) return e;
    if ((e = launch_kkt(KK_COLS, lanes_ka, lanes_kt, kr, s2)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(ev_join, s2)) != cudaSuccess) return e;
    if ((e = launch_kkt(KK_ROWS, lanes_ka, lanes_kt, kr, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, ev_join, 0)) != cudaSuccess) return e;
    if ((e = ndg_stages()) != cudaSuccess) return e;
    for (int k : {KK_FINAL, KK_APPLY, KK_END})
      if ((e = launch_kkt(k, lanes_ka, lanes_kt, kr, s)) != cudaSuccess) return e;
    return cudaSuccess;
  }
};

// The second capture stream and the fork / join events of a captured KKT block.
// The graph keeps the dependencies, not these objects, so they go with the capture.
struct Fork {
  cudaStream_t s2 = nullptr;
  cudaEvent_t f = nullptr, j = nullptr;
  cudaError_t make(Solve& sv) {
    cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    if (e == cudaSuccess) {
      sv.s2 = s2;
      sv.ev_fork = f;
      sv.ev_join = j;
    }
    return e;
  }
  ~Fork() {
    if (j) cudaEventDestroy(j);
    if (f) cudaEventDestroy(f);
    if (s2) cudaStreamDestroy(s2);
  }
};

static int check_inputs(const pdlp_csr* A, const void* b, const void* sense, const void* c,
                        const void* l, const void* u, const pdlp_params* p, const void* x_out,
                        const void* y_out, const pdlp_result* r) {
  if (!A || !r || !p) return fail(PDLP_ERR_INVALID_INPUT, "NULL problem, params or result");
  if (p->struct_size != sizeof(pdlp_params))
    return fail(PDLP_ERR_INVALID_INPUT, "pdlp_params.struct_size mismatch (use pdlp_default_params)");
  if (A->m < 0 || A->n < 1 || A->nnz < 0)
    return fail(PDLP_ERR_INVALID_INPUT, "need m >= 0, n >= 1, nnz >= 0");
  if (A->nnz >= (int64_t)INT32_MAX)
    return fail(PDLP_ERR_INVALID_INPUT, "nnz must be below 2^31 for one LP");
  if (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
    return fail(PDLP_ERR_INVALID_INPUT, "NULL CSR array");
  if ((A->m > 0 && (!b || !sense)) || !c || !l || !u || !x_out || (A->m > 0 && !y_out))
    return fail(PDLP_ERR_INVALID_INPUT, "NULL vector argument");
  if (!(p->tol > 0.0) || p->iter_limit < 0 || p->check_period < 1 || p->ruiz_iters < 0 ||
      !(p->time_limit_s > 0.0))
    return fail(PDLP_ERR_INVALID_INPUT, "invalid parameter value");
  if (p->precision != PDLP_FP64 && p->precision != PDLP_FP32 && p->precision != PDLP_FP32_BF16A)
    return fail(PDLP_ERR_INVALID_INPUT, "unknown precision mode");
  if (p->persistent < 0 || p->persistent > 2)
    return fail(PDLP_ERR_INVALID_INPUT, "persistent must be 0, 1 or 2");
  if (p->autotune != 0 && p->autotune != 1)
    return fail(PDLP_ERR_INVALID_INPUT, "autotune must be 0 or 1");
  if (p->tiles < 0 || p->tiles > 2) return fail(PDLP_ERR_INVALID_INPUT, "tiles must be 0, 1 or 2");
  if (p->bound_objective_rescaling != 0 && p->bound_objective_rescaling != 1)
    return fail(PDLP_ERR_INVALID_INPUT, "bound_objective_rescaling must be 0 or 1");
  if ((p->lanes_A && !valid_step_lanes(p->lanes_A)) || (p->lanes_AT && !valid_step_lanes(p->lanes_AT)))
    return fail(PDLP_ERR_INVALID_INPUT, "step lanes must be 0, 1, 2, 4, 8, 16 or 32");
  if ((p->lanes_kkt_A && !valid_lanes(p->lanes_kkt_A)) ||
      (p->lanes_kkt_AT && !valid_lanes(p->lanes_kkt_AT)))
    return fail(PDLP_ERR_INVALID_INPUT, "KKT lanes must be 0, 2, 4, 8, 16 or 32");
  if (p->persistent && (p->lanes_A == 1 || p->lanes_AT == 1))
    return fail(PDLP_ERR_INVALID_INPUT, "one lane per row needs persistent = 0");
  if (p->halpern != 0 && p->halpern != 1) return fail(PDLP_ERR_INVALID_INPUT, "halpern must be 0 or 1");
  if (p->halpern && !(p->halpern_reflection >= 0.0 && p->halpern_reflection <= 1.0))
    return fail(PDLP_ERR_INVALID_INPUT, "halpern_reflection must lie in [0, 1]");
  if (p->halpern && (p->persistent || p->tiles))
    return fail(PDLP_ERR_INVALID_INPUT, "halpern runs with persistent = 0 and tiles = 0 only");
  if (p->restart_metric != 0 && p->restart_metric != 1)
    return fail(PDLP_ERR_INVALID_INPUT, "restart_metric must be 0 or 1");
  if (p->restart_metric == 1 && (p->halpern || p->bound_objective_rescaling))
    return fail(PDLP_ERR_INVALID_INPUT,
                "restart_metric = 1 runs without halpern and bound_objective_rescaling");
  return PDLP_OK;
}

// Kernel timing request (pdlp_time_kernels): after the setup of a solve, each
// fused kernel is launched `reps` times back to back from a CUDA graph.
struct TimingReq {
  int reps;
  double* ms;     // [7] primal, dual, attempt (primal + dual), KKT pass over A, over A^T,
                  // one attempt inside the persistent kernel
  double* bytes;  // [7] algorithmic bytes per launch of the same kernels (per attempt for [5])
};

static int time_kernels_after_setup(Solve& sv, DevState* st, int mode, long long nnz,
                                    const TimingReq& tq, int count);

// Products of the device setup of one LP (rows A0-A3) into the buffers of a Bufs.
struct SetupOut {
  Mode mode;
  int scaled, fp32;
  double sca[8];  // ||c~||, ||q~||, ||c||, ||q||, max |K~|, ||x~_hint||, ||y~_hint||,
                  // columns with an infinite bound
  int lanes_a, lanes_t, lanes_ka, lanes_kt, th_a, th_t, nlong_a, nlong_t;
  int tiles, n_ta, n_tt;  // staged tile kernels built; their items over A and A^T
};

// Validation, canonical form, transpose, value format, scaling, iteration-space
// data and long-row lists of one LP.  forced_mode >= 0 skips the value-format
// choice; forced_lanes (A, A^T, KKT A, KKT A^T) overrides the lanes heuristic
// (a batch shares one kernel instantiation).
static int setup_lp(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                    const double* l, const double* u, const pdlp_params* p, const double* x0,
                    const double* y0, Bufs& bf, cudaStream_t s, bool no_alloc, int forced_mode,
                    const int* forced_lanes, SetupOut* so, const double* hx = nullptr,
                    const double* hy = nullptr,
                    const std::function<void(const char*)>& mark = [](const char*) {},
                    bool build_tiles = true) {
  const int m = A->m, n = A->n;
  const long long nnz = A->nnz;
  // ---- validation (A0 preconditions)
  SetupIn in{m, n, nnz, A->row_ptr, A->col, A->val, b, sense, c, l, u};
  CUDA_TRY(setup_validate(in, bf.flags2, s));
  g_launches += 3;
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, bf.flags2, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (err) {
    std::string msg = "invalid input:";
    if (err & ERR_ROWPTR) msg += " row_ptr";
    if (err & ERR_COL) msg += " column index";
    if (err & ERR_NONFINITE) msg += " non-finite value";
    if (err & ERR_SENSE) msg += " sense";
    if (err & ERR_BOUNDS) msg += " bounds";
    return fail(PDLP_ERR_INVALID_INPUT, msg);
  }
  mark("validate");
  // ---- A0, A1
  CUDA_TRY(setup_canonical(in, bf.a_ptr, bf.a_col, bf.a_val64, bf.q64, bf.row_kind, s));
  CUDA_TRY(setup_transpose(m, n, (int)nnz, bf.a_ptr, bf.a_col, bf.a_val64, bf.t_ptr, bf.t_col,
                           bf.t_val64, bf.tmp, s, no_alloc));
  g_launches += 10;
  mark("canonical + transpose");
  // ---- mode
  Mode mode = MODE_FP64;
  int bf16_exact = 0, all_one = 0;
  if (p->precision == PDLP_FP32) mode = MODE_FP32;
  if (forced_mode >= 0) {
    mode = (Mode)forced_mode;
  } else if (p->precision == PDLP_FP32_BF16A) {
    CUDA_TRY(setup_value_format(bf.a_val64, (int)nnz, bf.flags2, &bf16_exact, &all_one, s));
    ++g_launches;
    mode = all_one ? MODE_PAT : (bf16_exact ? MODE_BF16 : MODE_FP32);
  }
  const int scaled = (mode == MODE_FP64 || mode == MODE_FP32) ? 1 : 0;
  const int fp32 = mode != MODE_FP64;
  // ---- A2
  ScaleIn sc{m, n, bf.a_ptr, bf.a_col, bf.a_val64, bf.t_ptr, bf.t_col, bf.t_val64, p->ruiz_iters,
             p->pc_alpha, nnz};
  mark("value format");
  CUDA_TRY(setup_scaling(sc, bf.dr, bf.dc, bf.stat_r, bf.stat_c, s));
  g_launches += 2 + 2 * p->ruiz_iters + (p->pc_alpha >= 0 ? 2 : 0);
  mark("Ruiz + Pock-Chambolle");
  CUDA_TRY(setup_kkt_aux(m, n, bf.dr, bf.dc, l, u, bf.inv_dr, bf.inv_dc, bf.bflags, s));
  ++g_launches;
  if (mode != MODE_PAT) {
    const int vt = mode == MODE_FP64 ? 0 : (mode == MODE_FP32 ? 1 : 2);
    CUDA_TRY(setup_iter_values(vt, bf.a_ptr, bf.a_col, bf.a_val64, m, bf.dr, bf.dc, 1, scaled,
                               bf.a_valit, s));
    CUDA_TRY(setup_iter_values(vt, bf.t_ptr, bf.t_col, bf.t_val64, n, bf.dc, bf.dr, 0, scaled,
                               bf.t_valit, s));
    g_launches += 2;
  }
  VecIn vi{m, n, bf.dr, bf.dc, c, l, u, bf.q64, bf.row_kind, x0, y0, scaled, hx, hy};
  CUDA_TRY(setup_iter_vectors(vi, fp32, bf.c_it, bf.l_it, bf.u_it, bf.q_it, bf.tw, bf.sw, bf.x[0],
                              bf.y[0], bf.a_ptr, bf.a_col, bf.a_val64, bf.part_setup, bf.scalars, s));
  g_launches += 3;
  double sca[8];
  CUDA_TRY(cudaMemcpyAsync(sca, bf.scalars, sizeof(sca), cudaMemcpyDeviceToHost, s));
  mark("iteration values + vectors");
  // ---- launch shapes and long rows
  const double avg_a = m ? (double)nnz / m : 1.0, avg_t = (double)nnz / n;
  const double per_lane = mode == MODE_FP64 ? 8.0 : 4.0;
  const bool one_ok = mode != MODE_FP64 && !p->persistent;
  int lanes_a = p->lanes_A ? p->lanes_A : step_lanes(avg_a, per_lane, one_ok);
  int lanes_t = p->lanes_AT ? p->lanes_AT : step_lanes(avg_t, per_lane, one_ok);
  int lanes_ka = p->lanes_kkt_A ? p->lanes_kkt_A : auto_lanes(avg_a, 8.0);
  int lanes_kt = p->lanes_kkt_AT ? p->lanes_kkt_AT : auto_lanes(avg_t, 8.0);
  if (forced_lanes) {
    lanes_a = forced_lanes[0];
    lanes_t = forced_lanes[1];
    lanes_ka = forced_lanes[2];
    lanes_kt = forced_lanes[3];
  }
  const int th_a = long_thresh(lanes_a, lanes_ka);
  const int th_t = long_thresh(lanes_t, lanes_kt);
  int nlong_a = 0, nlong_t = 0;
  {
    const size_t R = (size_t)std::max(m, n) + 1;
    int* flags = bf.tmp;
    int* pos = flags + R;
    int* bsum = pos + R + 1;
    if (m > 0) CUDA_TRY(setup_long_rows(bf.a_ptr, m, th_a, flags, pos, bsum, bf.a_long, &nlong_a, s));
    CUDA_TRY(setup_long_rows(bf.t_ptr, n, th_t, flags, pos, bsum, bf.t_long, &nlong_t, s));
    g_launches += 10;
  }
  // work items of the staged tile kernels (float32 iterates)
  so->tiles = 0;
  so->n_ta = so->n_tt = 0;
  if (build_tiles && fp32 && p->tiles && !p->persistent && bf.tcap_t > 0) {
    int cnt[2] = {0, 0}, W = 0;
    const TileShape tsh = tile_shape(p->tiles);
    CUDA_TRY(setup_tiles(tsh, bf.a_ptr, m, nnz, nullptr, 1, bf.tmp, bf.ti_a, bf.tlp_a, bf.tlp_a + 2,
                         bf.tick_a, bf.tcap_a, cnt, &W, s));
    so->n_ta = cnt[0];
    CUDA_TRY(setup_tiles(tsh, bf.t_ptr, n, nnz, nullptr, 1, bf.tmp, bf.ti_t, bf.tlp_t, bf.tlp_t + 2,
                         bf.tick_t, bf.tcap_t, cnt, &W, s));
    so->n_tt = cnt[0];
    so->tiles = p->tiles;
    g_launches += 14;
  }
  CUDA_TRY(cudaStreamSynchronize(s));  // scalars
  so->mode = mode;
  so->scaled = scaled;
  so->fp32 = fp32;
  for (int k = 0; k < 8; ++k) so->sca[k] = sca[k];
  so->lanes_a = lanes_a;
  so->lanes_t = lanes_t;
  so->lanes_ka = lanes_ka;
  so->lanes_kt = lanes_kt;
  so->th_a = th_a;
  so->th_t = th_t;
  so->nlong_a = nlong_a;
  so->nlong_t = nlong_t;
  return PDLP_OK;
}

// ---------------------------------------------------------------- graph cache
// The CUDA graph of one check period captures the launch parameters by value
// (workspace pointers, grids, lanes, mode), so a caller that solves again into
// the same workspace with the same shape can relaunch the same executable
// graph.  Keyed by the bytes of those parameters and the device; a few entries,
// least recently used first out; never destroyed at process exit (the CUDA
// context may be gone by then).
struct GraphKey {
  int dev, mode, lanes[4], period, persist;
  IterRaw ir;
  KktRaw kr;
  bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  long long nodes;
  unsigned long long used;
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry>* g_graphs = new std::vector<GraphEntry>();
static unsigned long long g_graph_clock = 0;
constexpr size_t kGraphCacheSize = 8;

static GraphKey graph_key(const Solve& sv, int period) {
  GraphKey k;
  memset(&k, 0, sizeof(k));  // padding bytes take part in the comparison
  cudaGetDevice(&k.dev);
  k.mode = (int)sv.mode;
  k.lanes[0] = sv.lanes_a;
  k.lanes[1] = sv.lanes_t;
  k.lanes[2] = sv.lanes_ka;
  k.lanes[3] = sv.lanes_kt;
  k.period = period;
  k.persist = sv.persist_grid;
  memcpy(&k.ir, &sv.ir, sizeof(IterRaw));
  memcpy(&k.kr, &sv.kr, sizeof(KktRaw));
  return k;
}

// ---------------------------------------------------------------- launch-shape autotuner
// Lanes per row of the two step kernels, chosen by timing: every candidate
// (2, 4, 8, 16, 32 lanes; the primal kernel's over A^T, then the dual kernel's
// over A with the primal choice kept) runs a CUDA graph of kTuneReps whole step
// attempts on this LP with the state in dry mode (the kernels do all their work,
// the step decision is skipped, the current iterate is untouched), and the
// fastest is kept.  Results are cached per (device, mode, m, n, nnz) for the life
// of the process.
constexpr int kTuneReps = 16;
struct TuneKey {
  int dev, mode, count;
  long long m, n, nnz;
  bool one_lane;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, mode, count, m, n, nnz, one_lane) <
           std::tie(o.dev, o.mode, o.count, o.m, o.n, o.nnz, o.one_lane);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;

// Sets sv.lanes_t / sv.lanes_a; set_grids(lanes_t, lanes_a) applies a choice to
// the launch shapes (grids, batch maps); set_dry(on) switches the state(s)
// between dry mode (check_due 0, dry 1) and ready (check_due 1, dry 0).
template <typename SetGrids, typename SetDry>
static int autotune_lanes(Solve& sv, int count, bool tune_t, bool tune_a, bool one_lane,
                          SetGrids set_grids, SetDry set_dry) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  const TuneKey key{dev, (int)sv.mode, count, sv.m, sv.n, sv.nnz, one_lane};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      if (tune_t) sv.lanes_t = it->second.first;
      if (tune_a) sv.lanes_a = it->second.second;
      return set_grids(sv.lanes_t, sv.lanes_a);
    }
  }
  const cudaStream_t s = sv.s;
  int rc = set_dry(true);
  if (rc) return rc;
  cudaStream_t cs;
  CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t a, b;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  struct Free {
    cudaStream_t s;
    cudaEvent_t a, b;
    ~Free() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaStreamDestroy(s);
    }
  } fr{cs, a, b};
  auto time_one = [&](int which, double* out) -> int {
    Solve cap = sv;
    cap.s = cs;
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    // whole attempts whichever orientation is tuned: a kernel timed back to back with
    // itself runs from inputs it left in L2 and, alone, ranked 4 lanes over A ahead of 8 on
    // the covering LP, the reverse of their order inside attempts (27.0 against 22.2 us)
    (void)which;
    for (int i = 0; i < kTuneReps && ce == cudaSuccess; ++i) {
      ce = cap.iter(IK_PRIMAL);
      if (ce == cudaSuccess) ce = cap.iter(IK_DUAL);
    }
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (ce != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("tuning capture: ") + cudaGetErrorString(ce));
    CUDA_TRY(ee);
    cudaGraphExec_t ge;
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(ie);
    struct GFree {
      cudaGraphExec_t g;
      ~GFree() { cudaGraphExecDestroy(g); }
    } gf{ge};
    CUDA_TRY(cudaGraphLaunch(ge, s));  // warm
    CUDA_TRY(cudaEventRecord(a, s));
    CUDA_TRY(cudaGraphLaunch(ge, s));
    CUDA_TRY(cudaEventRecord(b, s));
    CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    *out = ms;
    g_launches += 2LL * 3 * kTuneReps;
    return PDLP_OK;
  };
  // one lane per row only for float32 iterates and the two-launch kernels
  static const int cand[6] = {1, 2, 4, 8, 16, 32};
  for (int which : {IK_PRIMAL, IK_DUAL}) {
    if ((which == IK_PRIMAL && !tune_t) || (which == IK_DUAL && !tune_a)) continue;
    double best = INFINITY;
    int best_l = which == IK_PRIMAL ? sv.lanes_t : sv.lanes_a;
    for (int L : cand) {
      if (L == 1 && !one_lane) continue;
      if (which == IK_PRIMAL) sv.lanes_t = L; else sv.lanes_a = L;
      if ((rc = set_grids(sv.lanes_t, sv.lanes_a)) != PDLP_OK) return rc;
      double ms = 0.0;
      if ((rc = time_one(which, &ms)) != PDLP_OK) return rc;
      if (ms < best) {
        best = ms;
        best_l = L;
      }
    }
    if (which == IK_PRIMAL) sv.lanes_t = best_l; else sv.lanes_a = best_l;
    if ((rc = set_grids(sv.lanes_t, sv.lanes_a)) != PDLP_OK) return rc;
  }
  if ((rc = set_dry(false)) != PDLP_OK) return rc;
  CUDA_TRY(cudaStreamSynchronize(s));
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {sv.lanes_t, sv.lanes_a};
  return PDLP_OK;
}

static int solve_device(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                        const double* l, const double* u, const pdlp_params* p, const double* x0,
                        const double* y0, double* x_out, double* y_out, pdlp_result* r,
                        const pdlp_diagnostics* dg, void* workspace, size_t ws_bytes,
                        cudaStream_t s, const TimingReq* tq = nullptr, bool no_alloc = false,
                        const double* hx = nullptr, const double* hy = nullptr) {
  const int m = A->m, n = A->n;
  const long long nnz = A->nnz;
  g_launches = 0;
  memset(r, 0, sizeof(*r));
  Bufs bf;
  Arena dry{nullptr, 0};
  const size_t need = carve(dry, bf, m, n, nnz, p->precision, p->restart_metric == 1);
  void* own_ws = nullptr;
  if (!workspace) {
    cudaError_t e = cudaMallocAsync(&own_ws, need, s);
    if (e != cudaSuccess) return fail(PDLP_ERR_OOM, std::string("workspace: ") + cudaGetErrorString(e));
    workspace = own_ws;
  } else if (ws_bytes < need || ((uintptr_t)workspace & 255)) {
    return fail(PDLP_ERR_OOM, "workspace smaller than pdlp_workspace_size or not 256-byte aligned");
  }
  struct Freer {
    void* p;
    cudaStream_t s;
    ~Freer() {
      if (p) cudaFreeAsync(p, s);
    }
  } freer{own_ws, s};
  Arena ar{(char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255), 0};
  carve(ar, bf, m, n, nnz, p->precision, p->restart_metric == 1);

  // no_alloc: nothing below creates a CUDA object or allocates memory (no events,
  // graphs, streams or pinned buffers); phases are timed with host clocks
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  if (!no_alloc) {
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventCreate(&e2));
  }
  struct EvFree {
    cudaEvent_t a, b, c;
    ~EvFree() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (c) cudaEventDestroy(c);
    }
  } evfree{e0, e1, e2};
  auto h0 = std::chrono::steady_clock::now(), h1 = h0, h2 = h0;
  if (!no_alloc) CUDA_TRY(cudaEventRecord(e0, s));

  // verbose >= 2: host-side phase times (the stream is synchronised at each mark)
  auto tmark = std::chrono::steady_clock::now();
  auto phase = [&](const char* what) {
    if (p->verbose < 2) return;
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    fprintf(stderr, "pdlp: %-28s %9.3f ms\n", what,
            1e3 * std::chrono::duration<double>(now - tmark).count());
    tmark = now;
  };
  phase("workspace");
  SetupOut so;
  {
    const int rc = setup_lp(A, b, sense, c, l, u, p, x0, y0, bf, s, no_alloc, -1, nullptr, &so, hx,
                            hy, phase);
    if (rc) return rc;
  }
  phase("long rows + scalars");
  const Mode mode = so.mode;
  const int scaled = so.scaled, fp32 = so.fp32;
  const double* sca = so.sca;
  const int lanes_a = so.lanes_a, lanes_t = so.lanes_t, lanes_ka = so.lanes_ka, lanes_kt = so.lanes_kt;
  const int th_a = so.th_a, th_t = so.th_t, nlong_a = so.nlong_a, nlong_t = so.nlong_t;
  const int MB = max_blocks();
  // float32 step kernels: one group of lanes per two rows, rows grid-strided;
  // float64 kernels (float64 steps, KKT passes): warp tiles of 32 rows
  const bool tiled = mode == MODE_FP64;
  // float32 step kernels: at most one wave of resident blocks (kStepBlocksPerSmF32 per
  // SM) including the long-row blocks, the short rows grid-strided; a second partial
  // wave would trail
  const int lt_blk = std::min(nlong_t, kMaxLongBlocks), la_blk = std::min(nlong_a, kMaxLongBlocks);
  const int wave = kStepBlocksPerSmF32 * device_sm_count();
  const int MBp = std::max(device_sm_count(), wave - lt_blk);
  const int MBd = std::max(device_sm_count(), wave - la_blk);
  const int gp_short = tiled ? grid_for(((long long)n + 31) / 32 * 32, MB)
                             : grid_for(((long long)n + 1) / 2 * lanes_t, MBp);
  const int gd_short = tiled ? grid_for(((long long)std::max(m, 1) + 31) / 32 * 32, MB)
                             : grid_for(((long long)std::max(m, 1) + 1) / 2 * lanes_a, MBd);
  const int gp = gp_short + std::min(nlong_t, kMaxLongBlocks);
  const int gd = gd_short + std::min(nlong_a, kMaxLongBlocks);
  const int ge = grid_for(std::max(m, n), MB);
  // KKT passes: up to six blocks per SM.  The passes over A and A^T run side by side on
  // two graph branches; measured per KKT block (prep, both passes, final, apply, end):
  // two blocks per SM 687 / 130 us on the energy system / covering LP, three 642 / 107,
  // four 615 / 109, six 615 / 100, eight 620 / 101 (the final reduction's longer partial
  // lists cost less than the passes gain from more warps in flight)
  const int KB = 6 * device_sm_count();
  const int gr_short = grid_for(((long long)std::max(m, 1) + 31) / 32 * 32, KB);
  const int gc_short = grid_for(((long long)n + 31) / 32 * 32, KB);
  const int gr = gr_short + std::min(nlong_a, kMaxLongBlocks);
  const int gc = gc_short + std::min(nlong_t, kMaxLongBlocks);

  IterRaw ir{};  // batch tables stay NULL: one LP
  ir.a_ptr = bf.a_ptr; ir.a_col = bf.a_col; ir.a_val = mode == MODE_PAT ? nullptr : bf.a_valit;
  ir.t_ptr = bf.t_ptr; ir.t_col = bf.t_col; ir.t_val = mode == MODE_PAT ? nullptr : bf.t_valit;
  ir.a_long = bf.a_long; ir.t_long = bf.t_long;
  ir.a_nlong = nlong_a; ir.t_nlong = nlong_t; ir.a_thresh = th_a; ir.t_thresh = th_t;
  ir.m = m; ir.n = n;
  ir.c = bf.c_it; ir.l = bf.l_it; ir.u = bf.u_it; ir.q = bf.q_it;
  ir.tw = scaled ? nullptr : bf.tw; ir.sw = scaled ? nullptr : bf.sw;
  ir.row_kind = bf.row_kind;
  for (int k = 0; k < 2; ++k) { ir.x[k] = bf.x[k]; ir.y[k] = bf.y[k]; }
  ir.sum_x = bf.sum_x; ir.sum_y = bf.sum_y;
  ir.part_p = bf.part_p; ir.part_d = bf.part_d;
  ir.grid_p_short = gp_short; ir.grid_p = gp; ir.grid_d_short = gd_short; ir.grid_d = gd;
  ir.st = bf.st;
  ir.count = 1;
  if (so.tiles) {
    int bp = 0, bd = 0;
    CUDA_TRY(tile_resident_mode(mode, so.tiles, &bp, &bd));
    ir.tile = so.tiles;
    ir.tslot = so.tiles == 1 ? kWarps : 1;
    ir.tt = TileSet{bf.ti_t, so.n_tt, bf.tlp_t, bf.tlp_t + 2, bf.tpart_t, bf.trow_t, bf.tlong_t, bf.tick_t};
    ir.ta = TileSet{bf.ti_a, so.n_ta, bf.tlp_a, bf.tlp_a + 2, bf.tpart_a, bf.trow_a, bf.tlong_a, bf.tick_a};
    tile_launch(so.tiles, so.n_tt, bp, &ir.grid_tt, &ir.work_tt);
    tile_launch(so.tiles, so.n_ta, bd, &ir.grid_ta, &ir.work_ta);
  }

  KktRaw kr{};
  kr.count = 1;
  kr.a_ptr = bf.a_ptr; kr.a_col = bf.a_col; kr.a_val64 = mode == MODE_PAT ? nullptr : bf.a_val64;
  kr.t_ptr = bf.t_ptr; kr.t_col = bf.t_col; kr.t_val64 = mode == MODE_PAT ? nullptr : bf.t_val64;
  kr.a_long = bf.a_long; kr.t_long = bf.t_long;
  kr.a_nlong = nlong_a; kr.t_nlong = nlong_t; kr.a_thresh = th_a; kr.t_thresh = th_t;
  kr.m = m; kr.n = n;
  kr.c = c; kr.l = l; kr.u = u; kr.q = bf.q64; kr.dr = bf.dr; kr.dc = bf.dc;
  kr.inv_dr = bf.inv_dr; kr.inv_dc = bf.inv_dc; kr.bflags = bf.bflags;
  kr.row_kind = bf.row_kind;
  for (int k = 0; k < 2; ++k) { kr.x[k] = bf.x[k]; kr.y[k] = bf.y[k]; }
  kr.sum_x = bf.sum_x; kr.sum_y = bf.sum_y;
  kr.XG = bf.XG; kr.Xl = bf.Xl; kr.YG = bf.YG; kr.Yl = bf.Yl; kr.XR = bf.XR; kr.YR = bf.YR;
  if (dg && dg->point_capacity > 0 && dg->check_points) {
    kr.chk_pts = dg->check_points;
    kr.chk_cap = dg->point_capacity;
  }
  // every column boxed: the primal ray is 0, only the dual ray is accumulated
  kr.rays = p->detect_infeasibility && p->terminate ? (sca[7] > 0.0 ? 2 : 1) : 0;
  kr.part_r = bf.part_r; kr.part_c = bf.part_c;
  kr.grid_r_short = gr_short; kr.grid_r = gr; kr.grid_c_short = gc_short; kr.grid_c = gc;
  kr.grid_e = ge;
  kr.scaled = scaled; kr.fp32 = fp32;
  kr.st = bf.st;
  if (p->restart_metric == 1) {
    kr.ndg_gx = bf.ndg_gx;
    kr.ndg_gy = bf.ndg_gy;
    kr.ndg = bf.ndg;
    kr.ndg_part = bf.ndg_part;
  }
  if (p->halpern) {
    // the Halpern iterate lives in the running-sum buffers (no averages in this variant)
    // and its anchor in the scaling statistics' (used only by the setup); the initial
    // KKT block sets both to the start
    ir.hx = kr.hx = bf.sum_x;
    ir.hy = kr.hy = bf.sum_y;
    ir.hax = kr.hax = bf.stat_c;
    ir.hay = kr.hay = bf.stat_r;
  }

  // ---- A3: initial state
  CUDA_TRY(cudaStreamSynchronize(s));  // scalars
  // Halpern variant: the constant step from the power-iteration estimate of ||K~||_2,
  // taken before any rescaling touches D_r and D_c (the KKT candidate buffers and
  // partials, not yet in use, are its scratch)
  double spectral = 0.0;
  if (p->halpern) {
    const int part_cap = kPartC * (max_blocks() + kMaxLongBlocks);
    PowIn pq{bf.a_ptr, bf.a_col, mode == MODE_PAT ? nullptr : bf.a_val64,
             bf.t_ptr, bf.t_col, mode == MODE_PAT ? nullptr : bf.t_val64,
             bf.a_long, bf.t_long, nlong_a, nlong_t, th_a, th_t, m, n, bf.dr, bf.dc};
    CUDA_TRY(setup_power_norm(pq, kPowerIters, (double*)bf.YG, (double*)bf.XG, bf.part_c,
                              part_cap, bf.part_r, &spectral, &g_launches, s));
  }
  // optional bound-objective rescaling: the objective by gamma = 1 + ||c~||, the
  // right-hand side and the bounds by beta = 1 + ||q~||; every scaled norm below is
  // taken in the rescaled problem
  double beta = 1.0, gamma = 1.0;
  if (p->bound_objective_rescaling) {
    gamma = 1.0 + sca[0];
    beta = 1.0 + sca[1];
    CUDA_TRY(setup_rescale(m, n, fp32, beta, gamma, bf.c_it, bf.l_it, bf.u_it, bf.q_it, bf.x[0],
                           bf.y[0], bf.dr, bf.dc, bf.inv_dr, bf.inv_dc, s));
    ++g_launches;
  }
  kr.ux = scaled ? 1.0 : beta;
  kr.uy = scaled ? 1.0 : gamma;
  DevState hs;
  memset(&hs, 0, sizeof(hs));
  const double nct = sca[0] / gamma, nqt = sca[1] / beta, kmax = sca[4];
  hs.omega = (nct > 1e-10 && nqt > 1e-10) ? nct / nqt : 1.0;
  // a primal-weight hint replaces the ||c~|| / ||q~|| estimate by the ratio of the
  // hint's own scaled norms (the balance the weight is meant to strike)
  const double nxh = sca[5] / beta, nyh = sca[6] / gamma;
  if ((hx || hy) && nxh > 1e-10 && nyh > 1e-10) hs.omega = nyh / nxh;
  hs.eta = kmax > 0.0 ? 1.0 / kmax : 1.0;
  if (p->fixed_eta > 0.0) hs.eta = p->fixed_eta;
  if (p->fixed_omega > 0.0) hs.omega = p->fixed_omega;
  if (p->halpern) {
    // a constant step, every step taken; the first epoch's coefficients (k = 0)
    hs.halpern = 1;
    hs.h_rho = p->halpern_reflection;
    hs.eta = spectral > 0.0 ? kHalpernEtaScale / spectral : 1.0;
    if (p->fixed_eta > 0.0) hs.eta = p->fixed_eta;
    hs.h_k = 0;
    hs.h_res = hs.h_r0 = INFINITY;
    halpern_coeffs(&hs);
  }
  hs.check_due = 1;
  hs.init_pending = 1;
  hs.prev_cand = INFINITY;
  hs.restart_metric = p->restart_metric;
  hs.ndg_last = INFINITY;
  hs.iter_limit = p->iter_limit;
  hs.period = p->check_period;
  hs.adaptive = p->adaptive_step && !p->halpern ? 1 : 0;
  hs.restarts_on = p->restarts ? 1 : 0;
  hs.terminate = p->terminate ? 1 : 0;
  hs.detect_inf = p->detect_infeasibility ? 1 : 0;
  hs.bar_skip = p->debug_skip_barrier ? 1 : 0;
  hs.spin_limit = p->debug_skip_barrier ? kSpinLimitTest : kSpinLimit;
  hs.tol = p->tol;
  hs.norm_c = sca[2];
  hs.norm_q = sca[3];
  hs.inv_omega = 1.0 / hs.omega;
  hs.tau_d = hs.eta / hs.omega;
  hs.sigma_d = hs.eta * hs.omega;
  hs.eta_f = (float)hs.eta;
  hs.omega_f = (float)hs.omega;
  hs.inv_omega_f = (float)hs.inv_omega;
  hs.tau_f = hs.eta_f * hs.inv_omega_f;
  hs.sigma_f = hs.eta_f * hs.omega_f;
  hs.pw_f = 0.0f;
  {
    const FacTable& ft = fac_table();
    CUDA_TRY(cudaMemcpyAsync(bf.fac, &ft, sizeof(FacTable), cudaMemcpyHostToDevice, s));
    hs.fac_dec = bf.fac->dec;
    hs.fac_inc = bf.fac->inc;
    hs.fac_dec_f = bf.fac->dec_f;
    hs.fac_inc_f = bf.fac->inc_f;
    hs.fac_n = kFacN;
  }
  if (dg && dg->attempt_capacity > 0 && dg->eta && dg->eta_bar && dg->accepted) {
    hs.tr_eta = dg->eta;
    hs.tr_eta_bar = dg->eta_bar;
    hs.tr_accepted = (signed char*)dg->accepted;
    hs.tr_cap = dg->attempt_capacity;
  }
  if (dg && dg->check_capacity > 0 && dg->restart && dg->omega) {
    hs.tr_restart = (signed char*)dg->restart;
    hs.tr_omega = dg->omega;
    hs.tr_check_cap = dg->check_capacity;
  }
  CUDA_TRY(cudaMemcpyAsync(bf.st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
  const size_t eb = fp32 ? 4 : 8;
  CUDA_TRY(cudaMemsetAsync(bf.sum_x, 0, eb * n, s));
  if (m) CUDA_TRY(cudaMemsetAsync(bf.sum_y, 0, eb * m, s));
  CUDA_TRY(cudaMemsetAsync(bf.Xl, 0, 8 * (size_t)n, s));
  if (m) CUDA_TRY(cudaMemsetAsync(bf.Yl, 0, 8 * (size_t)m, s));
  if (bf.ndg) CUDA_TRY(cudaMemsetAsync(bf.ndg, 0, sizeof(NdgState), s));

  Solve sv{m, n, nnz, mode, lanes_a, lanes_t, lanes_ka, lanes_kt, ir, kr, s, 0};
  // the autotuner creates a stream, events and graphs: never without allocation; the
  // staged tile kernels have no lanes to tune
  if (p->autotune && !no_alloc && !so.tiles && (!p->lanes_A || !p->lanes_AT) && p->iter_limit > 0) {
    auto set_grids = [&](int lt, int la) -> int {
      const int gps = tiled ? gp_short : grid_for(((long long)n + 1) / 2 * lt, MBp);
      const int gds = tiled ? gd_short : grid_for(((long long)std::max(m, 1) + 1) / 2 * la, MBd);
      sv.ir.grid_p_short = gps;
      sv.ir.grid_p = gps + std::min(nlong_t, kMaxLongBlocks);
      sv.ir.grid_d_short = gds;
      sv.ir.grid_d = gds + std::min(nlong_a, kMaxLongBlocks);
      return PDLP_OK;
    };
    auto set_dry = [&](bool on) -> int {
      static const int v[2][2] = {{1, 0}, {0, 1}};  // {check_due, dry}: ready, dry
      CUDA_TRY(cudaMemcpyAsync(&bf.st->check_due, &v[on][0], sizeof(int), cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(&bf.st->dry, &v[on][1], sizeof(int), cudaMemcpyHostToDevice, s));
      return PDLP_OK;
    };
    const bool one_lane_ok = !tiled && !p->persistent;
    const int rc = autotune_lanes(sv, 1, !p->lanes_AT, !p->lanes_A, one_lane_ok, set_grids,
                                  set_dry);
    if (rc) return rc;
  }
  if (p->persistent) {
    // the resident grid of the persistent kernel (probe launch with nothing to do:
    // the state says check_due, so every block returns at entry)
    // persistent = 2: one block (small LPs: the grid barrier is the block's barrier)
    const int want = p->persistent == 2 ? 1 : 0;
    if (p->persistent == 2) {
      // the one block holds the LP in shared memory when it fits (the 200 x 400
      // relaxations take 76 KB in float64), else it steps from global memory
      int dev = 0, optin = 0;
      CUDA_TRY(cudaGetDevice(&dev));
      CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      const SmemLayout L = smem_layout(m, n, nnz, mode == MODE_FP64 ? 8 : 4, mode != MODE_PAT,
                                       mode == MODE_BF16 || mode == MODE_PAT);
      if (L.bytes <= optin - kSmemStatic) {
        sv.ir.smem = L;
        // the order in which the block's threads take the columns and rows (longest
        // first), once per solve
        CUDA_TRY(setup_len_order(bf.t_ptr, n, bf.ord_t, s));
        if (m) CUDA_TRY(setup_len_order(bf.a_ptr, m, bf.ord_a, s));
        g_launches += m ? 2 : 1;
        sv.ir.ord_t = bf.ord_t;
        sv.ir.ord_a = bf.ord_a;
      }
    }
    int g = 0;
    cudaError_t e;
    switch (mode) {
      case MODE_FP64: e = launch_persist_fp64(sv.lanes_a, sv.lanes_t, sv.ir, 0, want, &g, s); break;
      case MODE_FP32: e = launch_persist_fp32(sv.lanes_a, sv.lanes_t, sv.ir, 0, want, &g, s); break;
      case MODE_BF16: e = launch_persist_bf16(sv.lanes_a, sv.lanes_t, sv.ir, 0, want, &g, s); break;
      default: e = launch_persist_pat(sv.lanes_a, sv.lanes_t, sv.ir, 0, want, &g, s); break;
    }
    ++g_launches;
    if (e != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("persistent kernel: ") + cudaGetErrorString(e));
    if (g > 4 * device_sm_count()) return fail(PDLP_ERR_CUDA, "persistent grid larger than its partial buffers");
    sv.persist_grid = g;
  }
  phase("state, tuning, probe");
  CUDA_TRY(sv.kkt_block());  // initial KKT and restart anchors
  phase("initial KKT");
  if (!no_alloc) {
    CUDA_TRY(cudaEventRecord(e1, s));
  } else {
    CUDA_TRY(cudaStreamSynchronize(s));
    h1 = std::chrono::steady_clock::now();
  }
  if (tq && !no_alloc) return time_kernels_after_setup(sv, bf.st, mode, nnz, *tq, 1);
  if (no_alloc) {
    // the same chunk of step attempts and KKT block, launched directly on the
    // caller's stream; the four-byte status is read into pageable memory
    if (p->iter_limit > 0) {
      static const int one[2] = {1, 1};
      const long long max_chunks = (p->iter_limit / p->check_period + 2) * 64 + 1024;
      bool forced = false;
      for (long long chunk = 0;; ++chunk) {
        CUDA_TRY(sv.period_steps(p->check_period));
        CUDA_TRY(sv.kkt_block());
        DevState h;
        CUDA_TRY(cudaMemcpyAsync(&h, bf.st, 16, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (h.status != 0) break;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - h1).count();
        if (!forced && el > p->time_limit_s) {
          CUDA_TRY(cudaMemcpyAsync(&bf.st->force_final, &one[0], sizeof(int), cudaMemcpyHostToDevice, s));
          CUDA_TRY(cudaMemcpyAsync(&bf.st->check_due, &one[1], sizeof(int), cudaMemcpyHostToDevice, s));
          forced = true;
        }
        if (chunk > max_chunks) return fail(PDLP_ERR_TIMEOUT, "iteration loop did not terminate");
      }
    }
    h2 = std::chrono::steady_clock::now();
  } else {

  // ---- iteration phase: graph of one check period
  DevState* hm = nullptr;  // pinned mirror of the first 16 bytes of the state, 2 slots
  CUDA_TRY(cudaMallocHost(&hm, 2 * sizeof(DevState)));
  struct HostFree {
    void* p;
    ~HostFree() { cudaFreeHost(p); }
  } hfree{hm};
  cudaEvent_t ev[2];
  CUDA_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
  struct EvFree2 {
    cudaEvent_t* e;
    ~EvFree2() {
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
    }
  } ev2{ev};
  cudaGraphExec_t gexec = nullptr;
  long long graph_nodes = 0;
  bool cached = false;
  const GraphKey gkey = graph_key(sv, p->check_period);
  if (p->iter_limit > 0) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (GraphEntry& e : *g_graphs)
      if (e.key == gkey) {
        gexec = e.exec;
        graph_nodes = e.nodes;
        e.used = ++g_graph_clock;
        cached = true;
        break;
      }
  }
  if (p->iter_limit > 0 && !cached) {
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct SFree {
      cudaStream_t s;
      ~SFree() { cudaStreamDestroy(s); }
    } csfree{cs};
    Solve cap = sv;
    cap.s = cs;
    Fork fork;
    CUDA_TRY(fork.make(cap));
    const long long before = g_launches;
    cudaGraph_t graph;
    if (sv.persist_grid > 0) {
      CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = cap.period_steps(p->check_period);
      if (ce == cudaSuccess) ce = cap.kkt_block();
      cudaError_t ee = cudaStreamEndCapture(cs, &graph);
      if (ce != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
      CUDA_TRY(ee);
    } else {
      // One check period: reset the attempt counter, then a while loop whose body is
      // kAttemptsPerBody step attempts (primal, dual, decision; dependent launches
      // between them) and whose condition the decision kernels set (go on until the
      // KKT check falls due), then the KKT block.  A body boundary costs a full
      // dependency, so a body holds several attempts; after the check falls due the
      // rest of the body returns at kernel entry.
      CUDA_TRY(cudaGraphCreate(&graph, 0));
      struct GDestroy {
        cudaGraph_t g;
        bool keep;
        ~GDestroy() {
          if (!keep) cudaGraphDestroy(g);
        }
      } gd{graph, false};
      cudaGraphConditionalHandle cond;
      CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
      cudaMemsetParams mp = {};
      mp.dst = &bf.st->loop_attempts;
      mp.value = 0;
      mp.elementSize = sizeof(int);
      mp.width = 1;
      mp.height = 1;
      cudaGraphNode_t reset;
      CUDA_TRY(cudaGraphAddMemsetNode(&reset, graph, nullptr, 0, &mp));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t loop;
      CUDA_TRY(cudaGraphAddNode(&loop, graph, &reset, nullptr, 1, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      cap.ir.cond = cond;
      cap.ir.loop_cap = 4 * p->check_period;
      CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = cudaSuccess;
      for (int a = 0; a < kAttemptsPerBody && ce == cudaSuccess; ++a) {
        ce = cap.iter(IK_PRIMAL);
        if (ce == cudaSuccess) ce = cap.iter(IK_DUAL);
      }
      cudaGraph_t body_out = body;
      cudaError_t ee = cudaStreamEndCapture(cs, &body_out);
      if (ce != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
      CUDA_TRY(ee);
      CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, graph, &loop, nullptr, 1,
                                             cudaStreamCaptureModeThreadLocal));
      ce = cap.kkt_block();
      cudaGraph_t main_out = graph;
      ee = cudaStreamEndCapture(cs, &main_out);
      if (ce != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
      CUDA_TRY(ee);
      gd.keep = true;
    }
    graph_nodes = g_launches - before;
    g_launches = before;
    cudaError_t ie = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(ie);
    std::lock_guard<std::mutex> lk(g_graph_mu);
    if (g_graphs->size() >= kGraphCacheSize) {
      auto old = std::min_element(g_graphs->begin(), g_graphs->end(),
                                  [](const GraphEntry& a, const GraphEntry& b) { return a.used < b.used; });
      cudaGraphExecDestroy(old->exec);
      g_graphs->erase(old);
    }
    g_graphs->push_back(GraphEntry{gkey, gexec, graph_nodes, ++g_graph_clock});
  }
  phase("graph capture + instantiate");

  const auto t_start = std::chrono::steady_clock::now();
  long long launched = 0, seen = 0;
  bool forced = false;
  const long long max_launches =
      (p->iter_limit / p->check_period + 2) * 64 + 1024;  // rejections re-run a chunk
  auto launch = [&]() -> cudaError_t {
    cudaError_t e = cudaGraphLaunch(gexec, s);
    if (e != cudaSuccess) return e;
    g_launches += graph_nodes;
    e = cudaMemcpyAsync(&hm[launched & 1], bf.st, 16, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev[launched & 1], s);
    ++launched;
    return e;
  };
  if (p->iter_limit > 0) {
    CUDA_TRY(launch());
    while (true) {
      if (launched - seen < 2) CUDA_TRY(launch());
      CUDA_TRY(cudaEventSynchronize(ev[seen & 1]));
      const DevState& h = hm[seen & 1];
      ++seen;
      if (h.status != 0) break;
      if (p->verbose)
        fprintf(stderr, "pdlp: chunk %lld iters %lld\n", seen, (long long)h.iters);
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
      if (!forced && el > p->time_limit_s) {
        // ask for a final check: the next chunk's steps are skipped and its KKT block terminates
        static const int one[2] = {1, 1};
        CUDA_TRY(cudaMemcpyAsync(&bf.st->force_final, &one[0], sizeof(int), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(&bf.st->check_due, &one[1], sizeof(int), cudaMemcpyHostToDevice, s));
        forced = true;
      }
      if (launched > max_launches) return fail(PDLP_ERR_TIMEOUT, "iteration loop did not terminate");
    }
  }
  CUDA_TRY(cudaStreamSynchronize(s));  // drain the chunk launched behind the terminating one
  phase("iterations");
  CUDA_TRY(cudaEventRecord(e2, s));
  }  // graph-driven iteration phase
  // ---- A11: outputs
  CUDA_TRY(launch_output(kr, x_out, m ? y_out : nullptr, dg ? dg->x_cur : nullptr,
                         dg && m ? dg->y_cur : nullptr, dg ? dg->x_avg : nullptr,
                         dg && m ? dg->y_avg : nullptr, s));
  ++g_launches;
  DevState fs;
  CUDA_TRY(cudaMemcpyAsync(&fs, bf.st, sizeof(fs), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  float ms_setup = 0.f, ms_solve = 0.f;
  if (!no_alloc) {
    cudaEventElapsedTime(&ms_setup, e0, e1);
    cudaEventElapsedTime(&ms_solve, e1, e2);
  } else {
    ms_setup = (float)(1e3 * std::chrono::duration<double>(h1 - h0).count());
    ms_solve = (float)(1e3 * std::chrono::duration<double>(h2 - h1).count());
  }

  if (fs.status == kStatusWaitFailed)
    return fail(PDLP_ERR_TIMEOUT,
                "a bounded wait of a step kernel gave up (a grid barrier of the persistent kernel "
                "or a staged copy of the tile kernels)");
  r->status = p->iter_limit == 0 ? PDLP_ITER_LIMIT : fs.status;
  r->precision_used = mode == MODE_FP64 ? PDLP_FP64
                      : mode == MODE_FP32 ? PDLP_FP32
                      : mode == MODE_BF16 ? PDLP_USED_BF16
                                          : PDLP_USED_PATTERN;
  r->lanes_A = sv.lanes_a;
  r->lanes_AT = sv.lanes_t;
  r->tiles = sv.ir.tile;
  r->persistent_form = p->persistent == 0 ? 0 : p->persistent == 1 ? 1 : sv.ir.smem.bytes > 0 ? 3 : 2;
  r->spectral_norm = spectral;
  r->iters = fs.iters;
  r->attempts = fs.attempts;
  r->restarts = fs.restarts;
  r->kkt_checks = fs.checks;
  const int k = fs.used_avg ? 1 : 0;
  r->used_average = k;
  r->primal_obj = fs.pobj[k];
  r->dual_obj = fs.dobj[k];
  r->rel_primal_res = fs.relp[k];
  r->rel_dual_res = fs.reld[k];
  r->rel_gap = fs.relgap[k];
  r->rel_kkt = std::max(r->rel_primal_res, std::max(r->rel_dual_res, r->rel_gap));
  r->eta = fs.eta;
  r->omega = fs.omega;
  const bool cert = fs.status == PDLP_PRIMAL_INFEASIBLE || fs.status == PDLP_DUAL_INFEASIBLE;
  r->ray_obj = cert ? fs.ray_obj : NAN;
  r->ray_res = cert ? fs.ray_res : NAN;
  r->setup_s = ms_setup * 1e-3;
  r->solve_s = ms_solve * 1e-3;
  // the while-loop graph was counted with one attempt per launch; its other
  // attempts ran as further iterations of the loop body (three kernels each)
  if (!no_alloc && sv.persist_grid == 0 && p->iter_limit > 0)
    g_launches += 3LL * kAttemptsPerBody *
                  std::max(0LL, (fs.attempts + kAttemptsPerBody - 1) / kAttemptsPerBody - fs.checks);
  r->kernel_launches = g_launches;
  return PDLP_OK;
}

static int time_kernels_after_setup(Solve& sv, DevState* st, int mode, long long nnz,
                                    const TimingReq& tq, int count) {
  const cudaStream_t s = sv.s;
  const int m = sv.m, n = sv.n;
  // the state every timing starts from (one per LP of a batch): every step attempt stays
  // live (no KKT check falls due, no iteration limit), and a step kind repeated on its own
  // can drive the iterate out of range (dual steps without primal steps grow y without
  // bound) -- a NaN ends the iteration at the next decision, after which the kernels
  // return at entry -- so each timed launch starts from this state
  std::vector<DevState> st0((size_t)count);
  CUDA_TRY(cudaMemcpyAsync(st0.data(), st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (DevState& h : st0) {
    h.period = 1 << 30;
    h.iter_limit = 1LL << 62;
  }
  static const int zero = 0;
  cudaStream_t cs;
  CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct SFree {
    cudaStream_t s;
    ~SFree() { cudaStreamDestroy(s); }
  } sfree{cs};
  cudaEvent_t a, b;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  struct EFree {
    cudaEvent_t a, b;
    ~EFree() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } efree{a, b};
  Solve cap = sv;
  cap.s = cs;
  Fork fork;
  CUDA_TRY(fork.make(cap));
  // which: 0 primal, 1 dual, 2 attempt, 3 KKT rows, 4 KKT cols, 5 persistent, 6 KKT block
  auto time_one = [&](int which, double* out_ms) -> int {
    cudaGraph_t g;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    if (which == 5) ce = cap.persist(tq.reps);  // reps attempts inside one launch
    for (int i = 0; i < tq.reps && ce == cudaSuccess && which != 5; ++i) {
      if (which == 0 || which == 2) ce = cap.iter(IK_PRIMAL);
      if (ce == cudaSuccess && (which == 1 || which == 2)) ce = cap.iter(IK_DUAL);
      if (which == 3) ce = launch_kkt(KK_ROWS, sv.lanes_ka, sv.lanes_kt, sv.kr, cs);
      if (which == 4) ce = launch_kkt(KK_COLS, sv.lanes_ka, sv.lanes_kt, sv.kr, cs);
      if (which == 6) {
        // check_due is 0 or 1, so setting its low byte (little endian) makes it 1
        ce = cudaMemsetAsync(&st->check_due, 1, 1, cs);
        if (ce == cudaSuccess) ce = cap.kkt_block();
      }
    }
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    if (ce != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    CUDA_TRY(ee);
    cudaGraphExec_t ge;
    cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(ie);
    struct GFree {
      cudaGraphExec_t g;
      ~GFree() { cudaGraphExecDestroy(g); }
    } gfree{ge};
    std::vector<DevState> run(st0);
    for (DevState& h : run) h.check_due = (which == 3 || which == 4) ? 1 : 0;
    const size_t sb = sizeof(DevState) * run.size();
    CUDA_TRY(cudaMemcpyAsync(st, run.data(), sb, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(ge, s));  // warm
    CUDA_TRY(cudaMemcpyAsync(st, run.data(), sb, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaEventRecord(a, s));
    CUDA_TRY(cudaGraphLaunch(ge, s));
    CUDA_TRY(cudaEventRecord(b, s));
    CUDA_TRY(cudaStreamSynchronize(s));  // `run` is read by the copies above
    CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    *out_ms = (double)ms / tq.reps;
    g_launches += which == 5 ? 2 : 2LL * tq.reps * (which == 2 ? 2 : which == 6 ? 6 : 1);
    return PDLP_OK;
  };
  int rc;
  // the primal step and the whole attempt repeat what a solve does; the dual half-step
  // is their difference (repeated on its own it would step y away without bound)
  if ((rc = time_one(0, &tq.ms[0])) != PDLP_OK) return rc;
  if ((rc = time_one(2, &tq.ms[2])) != PDLP_OK) return rc;
  tq.ms[1] = tq.ms[2] - tq.ms[0];
  if (sv.persist_grid > 0) {
    if ((rc = time_one(5, &tq.ms[5])) != PDLP_OK) return rc;
  } else {
    tq.ms[5] = 0.0;
  }
  for (int w = 3; w < 5; ++w)
    if ((rc = time_one(w, &tq.ms[w])) != PDLP_OK) return rc;
  // whole KKT blocks last: they move the restart anchors and the iterate (one LP: the
  // graph sets that LP's check flag before each block; a batch's block is not timed)
  if (count == 1) {
    if ((rc = time_one(6, &tq.ms[6])) != PDLP_OK) return rc;
  } else {
    tq.ms[6] = 0.0;
  }
  for (int k = 0; k < count; ++k)
    CUDA_TRY(cudaMemcpyAsync(&st[k].check_due, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  // algorithmic bytes per launch: every array the kernel needs, each element once
  // (gathered vectors counted once, not once per nonzero)
  const double M = m, N = n, Z = (double)nnz;
  const double sx = mode == MODE_FP64 ? 8 : 4;
  const double sv_b = mode == MODE_FP64 ? 8 : mode == MODE_FP32 ? 4 : mode == MODE_BF16 ? 2 : 0;
  const double impl = (mode == MODE_BF16 || mode == MODE_PAT) ? 1 : 0;
  const double val64 = mode == MODE_PAT ? 0 : 8;
  // primal: row_ptr, col, values; y gathered; x (pair) read, c, l, u (+ tw), pair write, sum r/w
  tq.bytes[0] = 4 * (N + 1) + Z * (4 + sv_b) + M * sx + N * sx * (2 + 3 + impl + 2 + 2);
  // dual: row_ptr, col, values; x pairs gathered; y, q (+ sw), row kind, y write, sum r/w
  tq.bytes[1] = 4 * (M + 1) + Z * (4 + sv_b) + N * 2 * sx + M * (sx * (1 + 1 + impl + 1 + 2) + 1);
  tq.bytes[2] = tq.bytes[0] + tq.bytes[1];
  // certificate terms: the dual ray (rays >= 1) and the primal ray (rays == 2)
  const double ry = sv.kr.rays >= 1 ? 8 : 0, rx = sv.kr.rays == 2 ? 8 : 0;
  // KKT over A: row_ptr, col, float64 values (none for a pattern); x candidates
  // gathered (and the primal ray);
  // q, D_r, 1/D_r, kind, y candidates (and the dual ray), y anchor
  tq.bytes[3] = 4 * (M + 1) + Z * (4 + val64) + N * (16 + rx) + M * (8 + 8 + 8 + 1 + 16 + ry + 8);
  // KKT over A^T: row_ptr, col, values; y candidates gathered (and the dual ray); c, l, u,
  // D_c, 1/D_c, bound flags, x candidates (and the primal ray), x anchor
  tq.bytes[4] = 4 * (N + 1) + Z * (4 + val64) + M * (16 + ry) + N * (8 + 16 + 8 + 8 + 1 + 16 + rx + 8);
  // one attempt of the persistent kernel: the primal and dual bytes
  tq.bytes[5] = tq.bytes[2];
  tq.bytes[6] = tq.bytes[3] + tq.bytes[4];
  return PDLP_OK;
}

// ---------------------------------------------------------------- batches
// Many LPs solved together: each LP is set up with setup_lp into a per-LP
// scratch workspace, then exported into one block-diagonal problem (global row
// and column numbering, global vectors).  The step and KKT kernels run over all
// LPs in one launch each; every block belongs to one LP (launch tables) and
// each LP keeps its own device state, step size, primal weight, restarts and
// termination.  One graph holds check_period attempts plus the KKT block for
// the whole batch.
struct LpShape {
  int m, n;
  long long nnz;
  long long R, C, Z;  // global first row, column, nonzero
};

// blocks of one LP in a launch map: proportional to its rows, at least one,
// never more than its rows need
static void build_map(const std::vector<LpShape>& sh, bool over_cols, int lanes, bool tiled,
                      const std::vector<int>& nlong, const std::vector<int>& long0, long long total_rows,
                      int budget, std::vector<int>& tab, int* grid) {
  const int K = (int)sh.size();
  std::vector<int> nshort(K), nblk(K), blk0(K), row0(K), nrows(K);
  long long g = 0;
  for (int k = 0; k < K; ++k) {
    const long long rows = over_cols ? sh[k].n : sh[k].m;
    const long long need = tiled ? (rows + 255) / 256 : ((rows + 1) / 2 * lanes + kBlock - 1) / kBlock;
    long long share = total_rows > 0 ? (long long)((double)budget * (double)rows / (double)total_rows) : 1;
    share = std::max(1LL, std::min(share, std::max(1LL, need)));
    nshort[k] = (int)share;
    nblk[k] = nshort[k] + std::min(nlong[k], kMaxLongBlocks);
    blk0[k] = (int)g;
    g += nblk[k];
    row0[k] = (int)(over_cols ? sh[k].C : sh[k].R);
    nrows[k] = (int)rows;
  }
  *grid = (int)g;
  tab.assign((size_t)g + 7 * (size_t)K, 0);
  for (int k = 0; k < K; ++k)
    for (int b = 0; b < nblk[k]; ++b) tab[blk0[k] + b] = k;
  int* t = tab.data() + g;
  for (int k = 0; k < K; ++k) {
    t[0 * K + k] = blk0[k];
    t[1 * K + k] = nshort[k];
    t[2 * K + k] = nblk[k];
    t[3 * K + k] = row0[k];
    t[4 * K + k] = nrows[k];
    t[5 * K + k] = long0[k];
    t[6 * K + k] = nlong[k];
  }
}

static Tables tables_at(int* dev, int grid, int K) {
  Tables t;
  t.blk_lp = dev;
  t.blk0 = dev + grid;
  t.nshort = dev + grid + K;
  t.nblk = dev + grid + 2 * K;
  t.row0 = dev + grid + 3 * K;
  t.nrows = dev + grid + 4 * K;
  t.long0 = dev + grid + 5 * K;
  t.nlong = dev + grid + 6 * K;
  return t;
}

// device_inputs: the LPs' arrays and the outputs are device buffers and the work runs
// on `user_stream`; otherwise host buffers, uploaded on a stream of the call's own.
static int solve_batch(int count, const pdlp_csr* const* A, const double* const* b,
                       const char* const* sense, const double* const* c, const double* const* l,
                       const double* const* u, const pdlp_params* p, double* const* x_out,
                       double* const* y_out, pdlp_result* res, const TimingReq* tq = nullptr,
                       bool device_inputs = false, cudaStream_t user_stream = nullptr) {
  if (p->bound_objective_rescaling)
    return fail(PDLP_ERR_INVALID_INPUT, "bound_objective_rescaling is for single LPs, not batches");
  if (p->halpern) return fail(PDLP_ERR_INVALID_INPUT, "halpern is for single LPs, not batches");
  if (p->restart_metric)
    return fail(PDLP_ERR_INVALID_INPUT, "restart_metric = 1 is for single LPs, not batches");
  if (p->persistent == 2)
    return fail(PDLP_ERR_INVALID_INPUT, "persistent = 2 (one block) is for single LPs, not batches");
  g_launches = 0;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = user_stream;
  if (!device_inputs) CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct SFree {
    cudaStream_t s;
    bool own;
    ~SFree() {
      if (own) cudaStreamDestroy(s);
    }
  } sfree{s, !device_inputs};
  // ---- shapes and global numbering
  std::vector<LpShape> sh(count);
  long long M = 0, N = 0, Z = 0;
  for (int k = 0; k < count; ++k) {
    sh[k] = {A[k]->m, A[k]->n, A[k]->nnz, M, N, Z};
    M += A[k]->m;
    N += A[k]->n;
    Z += A[k]->nnz;
  }
  if (M >= INT32_MAX || N >= INT32_MAX || Z >= INT32_MAX)
    return fail(PDLP_ERR_INVALID_INPUT, "a batch must have fewer than 2^31 rows, columns and nonzeros");
  // ---- one mode and one set of lanes for the whole batch (one kernel instantiation);
  // FP32_BF16A settles on the pattern / bfloat16 form after the canonical form, on the device
  int mode = p->precision == PDLP_FP64 ? MODE_FP64 : MODE_FP32;
  const double per_lane = mode == MODE_FP64 ? 8.0 : 4.0;
  const double avg_a = M ? (double)Z / (double)M : 1.0, avg_t = N ? (double)Z / (double)N : 1.0;
  // a float32 batch whose step data is well beyond L2 streams from HBM, where the dual
  // kernel gathers the (x', dx) pairs from DRAM: a quarter of the lanes per row (four
  // times the rows per warp in flight) measured faster there (256 covering sub-LPs,
  // 142M nonzeros: 629 us per dual half-step against 815 us with 8 lanes, the
  // iteration phase 0.295 against 0.343 s), while L2-resident problems keep the count
  // that wins on them (float64 batches were not measured and keep theirs)
  const double step_bytes = 2.0 * (double)Z * 8.0 + 40.0 * (double)(M + N);
  const double per_lane_a =
      mode != MODE_FP64 && step_bytes > 256e6 ? 4.0 * per_lane : per_lane;
  // one lane per row: float32 and the two-launch kernels only
  const bool one_ok = mode != MODE_FP64 && !p->persistent;
  int lanes[4] = {p->lanes_A ? p->lanes_A : step_lanes(avg_a, per_lane_a, one_ok),
                  p->lanes_AT ? p->lanes_AT : step_lanes(avg_t, per_lane, one_ok),
                  p->lanes_kkt_A ? p->lanes_kkt_A : auto_lanes(avg_a, 8.0),
                  p->lanes_kkt_AT ? p->lanes_kkt_AT : auto_lanes(avg_t, 8.0)};
  const size_t eb = mode == MODE_FP64 ? 8 : 4;
  const size_t vb = mode == MODE_FP64 ? 8 : 4;  // bound: bfloat16 (2) / pattern (0) fit
  const long long RM = std::max(M, N) + 1;
  const size_t tmp_ints = std::max(std::max(transpose_tmp_ints((int)M, (int)N, Z),
                                            2 * (size_t)RM + scan_tmp_ints(RM)),
                                   tile_tmp_ints((int)std::max(M, N)));
  // ---- global arrays
  struct G {
    int *a_ptr, *a_col, *t_ptr, *t_col, *a_long, *t_long, *tabA, *tabT;
    double *a_val64, *t_val64, *q64, *dr, *dc, *inv_dr, *inv_dc, *Xl, *Yl;
    double2 *XG, *YG;
    double *XR, *YR;
    double *c64, *l64, *u64, *part_p, *part_d, *part_r, *part_c, *x_out, *y_out;
    void *a_valit, *t_valit, *c_it, *l_it, *u_it, *q_it, *tw, *sw, *x[2], *y[2], *sum_x, *sum_y;
    unsigned char *row_kind, *bflags;
    DevState* st;
    FacTable* fac;
    // batched setup: the batch in global numbering as the callers gave it, scratch
    int64_t *rp_in, *rp_up;
    int* col_in;
    double *val_in, *b_in, *stat_r, *stat_c, *part_setup, *scalars, *lpsca;
    char* sense_in;
    int *tmp, *flags2, *errs, *lb_a, *lb_t;
    BatchLp* lps;
    // staged tile kernels over the block-diagonal A and A^T
    TileItem *ti_a, *ti_t;
    float2 *tpart_a, *tpart_t, *trow_a, *trow_t, *tlong_a, *tlong_t;
    int *tick_a, *tick_t, *tlp_a, *tlp_t, *row0_a, *row0_t;
  } g{};
  const bool use_tiles = mode != MODE_FP64 && p->tiles && !p->persistent;
  const TileShape tsh = tile_shape(p->tiles);
  const size_t tcap_a = use_tiles ? tile_item_cap(tsh, (int)M, Z, count) : 0;
  const size_t tcap_t = use_tiles ? tile_item_cap(tsh, (int)N, Z, count) : 0;
  const size_t tslot = p->tiles == 1 ? kWarps : 1;  // partials per slot
  // long rows and launch maps need the setup first: upper bounds here
  const int MB = max_blocks();
  const int budget = 4 * MB;
  const size_t gmax = (size_t)budget + (size_t)count * (kMaxLongBlocks + 2);
  auto lay = [&](Arena& ar) {
    g.fac = (FacTable*)ar.take(sizeof(FacTable));
    g.a_ptr = (int*)ar.take(4 * (M + 1));
    g.t_ptr = (int*)ar.take(4 * (N + 1));
    g.a_col = (int*)ar.take(4 * Z);
    g.t_col = (int*)ar.take(4 * Z);
    g.a_val64 = (double*)ar.take(8 * Z);
    g.t_val64 = (double*)ar.take(8 * Z);
    g.a_valit = ar.take(vb * Z);
    g.t_valit = ar.take(vb * Z);
    for (double** v : {&g.q64, &g.dr, &g.inv_dr, &g.Yl, &g.y_out, &g.b_in, &g.stat_r})
      *v = (double*)ar.take(8 * M);
    g.YG = (double2*)ar.take(16 * M);
    g.XG = (double2*)ar.take(16 * N);
    g.YR = (double*)ar.take(8 * M);
    g.XR = (double*)ar.take(8 * N);
    for (double** v : {&g.dc, &g.inv_dc, &g.Xl, &g.c64, &g.l64, &g.u64, &g.x_out, &g.stat_c})
      *v = (double*)ar.take(8 * N);
    g.row_kind = (unsigned char*)ar.take(M);
    g.sense_in = (char*)ar.take(M);
    g.bflags = (unsigned char*)ar.take(N);
    for (void** v : {&g.c_it, &g.l_it, &g.u_it, &g.tw, &g.sum_x}) *v = ar.take(eb * N);
    for (void** v : {&g.q_it, &g.sw, &g.sum_y}) *v = ar.take(eb * M);
    for (int k = 0; k < 2; ++k) {
      g.x[k] = ar.take(2 * eb * N);
      g.y[k] = ar.take(eb * M);
    }
    g.part_p = (double*)ar.take(8 * gmax);
    g.part_d = (double*)ar.take(8 * 2 * gmax);
    g.part_r = (double*)ar.take(8 * kPartR * gmax);
    g.part_c = (double*)ar.take(8 * kPartC * gmax);
    g.a_long = (int*)ar.take(4 * (M + 1));
    g.t_long = (int*)ar.take(4 * (N + 1));
    g.tabA = (int*)ar.take(4 * (gmax + 7 * (size_t)count));
    g.tabT = (int*)ar.take(4 * (gmax + 7 * (size_t)count));
    g.st = (DevState*)ar.take(sizeof(DevState) * count);
    g.rp_in = (int64_t*)ar.take(8 * (M + 1));
    g.rp_up = device_inputs ? nullptr : (int64_t*)ar.take(8 * (M + (size_t)count));
    g.col_in = (int*)ar.take(4 * Z);
    g.val_in = (double*)ar.take(8 * Z);
    g.part_setup = (double*)ar.take(8 * setup_part_doubles((int)M, (int)N));
    g.scalars = (double*)ar.take(8 * 8);
    g.lpsca = (double*)ar.take(8 * 8 * (size_t)count);
    g.tmp = (int*)ar.take(4 * tmp_ints);
    g.flags2 = (int*)ar.take(16);
    g.errs = (int*)ar.take(4 * (size_t)count);
    g.lb_a = (int*)ar.take(4 * ((size_t)count + 1));
    g.lb_t = (int*)ar.take(4 * ((size_t)count + 1));
    g.lps = (BatchLp*)ar.take(sizeof(BatchLp) * (size_t)count);
    if (use_tiles) {
      g.ti_a = (TileItem*)ar.take(sizeof(TileItem) * tcap_a);
      g.ti_t = (TileItem*)ar.take(sizeof(TileItem) * tcap_t);
      g.tpart_a = (float2*)ar.take(8 * tslot * tcap_a);
      g.tpart_t = (float2*)ar.take(8 * tslot * tcap_t);
      for (float2** v : {&g.trow_a, &g.tlong_a}) *v = (float2*)ar.take(8 * tcap_a);
      for (float2** v : {&g.trow_t, &g.tlong_t}) *v = (float2*)ar.take(8 * tcap_t);
      g.tick_a = (int*)ar.take(4 * tcap_a);
      g.tick_t = (int*)ar.take(4 * tcap_t);
      for (int** v : {&g.tlp_a, &g.tlp_t}) *v = (int*)ar.take(4 * 2 * ((size_t)count + 1));
      for (int** v : {&g.row0_a, &g.row0_t}) *v = (int*)ar.take(4 * ((size_t)count + 1));
    }
  };
  Arena gdry{nullptr, 0};
  lay(gdry);
  const size_t total = gdry.off + 256;
  void* dev = nullptr;
  {
    cudaError_t e = cudaMallocAsync(&dev, total, s);
    if (e != cudaSuccess) return fail(PDLP_ERR_OOM, std::string("batch buffers: ") + cudaGetErrorString(e));
  }
  struct DevFree {
    void* p;
    cudaStream_t s;
    ~DevFree() {
      cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } dfree{dev, s};
  Arena gar{(char*)dev, 0};
  lay(gar);
  const FacTable& ft = fac_table();
  CUDA_TRY(cudaMemcpyAsync(g.fac, &ft, sizeof(FacTable), cudaMemcpyHostToDevice, s));
  // ---- the batch in global numbering (A0 preconditions checked per LP on the way)
  std::vector<BatchLp> hl(count);
  for (int k = 0; k < count; ++k) {
    const LpShape& q = sh[k];
    BatchLp& L = hl[k];
    L.m = q.m;
    L.n = q.n;
    L.nnz = q.nnz;
    L.R = q.R;
    L.C = q.C;
    L.Z = q.Z;
    if (device_inputs) {
      L.rp = A[k]->row_ptr;
      L.col = A[k]->col;
      L.val = A[k]->val;
      L.b = b[k];
      L.sense = sense[k];
      L.c = c[k];
      L.l = l[k];
      L.u = u[k];
    } else {
      // host arrays: uploaded straight to their places in the global arrays (row
      // pointers to a staging array, one slot more per LP); the ingest kernel then
      // checks them and shifts the indices in place
      int64_t* rp = g.rp_up + q.R + k;
      auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
      };
      CUDA_TRY(up(rp, A[k]->row_ptr, 8 * ((size_t)q.m + 1)));
      CUDA_TRY(up(g.col_in + q.Z, A[k]->col, 4 * (size_t)q.nnz));
      CUDA_TRY(up(g.val_in + q.Z, A[k]->val, 8 * (size_t)q.nnz));
      CUDA_TRY(up(g.b_in + q.R, b[k], 8 * (size_t)q.m));
      CUDA_TRY(up(g.sense_in + q.R, sense[k], (size_t)q.m));
      CUDA_TRY(up(g.c64 + q.C, c[k], 8 * (size_t)q.n));
      CUDA_TRY(up(g.l64 + q.C, l[k], 8 * (size_t)q.n));
      CUDA_TRY(up(g.u64 + q.C, u[k], 8 * (size_t)q.n));
      L.rp = rp;
      L.col = g.col_in + q.Z;
      L.val = g.val_in + q.Z;
      L.b = g.b_in + q.R;
      L.sense = g.sense_in + q.R;
      L.c = g.c64 + q.C;
      L.l = g.l64 + q.C;
      L.u = g.u64 + q.C;
    }
  }
  if (!device_inputs) CUDA_TRY(cudaStreamSynchronize(s));
  const double upload_s =
      device_inputs ? 0.0 : std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  CUDA_TRY(cudaMemcpyAsync(g.lps, hl.data(), sizeof(BatchLp) * (size_t)count, cudaMemcpyHostToDevice, s));
  {
    long long mx = 1;
    for (const LpShape& q : sh) mx = std::max(mx, std::max((long long)q.m + 1, std::max(q.nnz, (long long)q.n)));
    CUDA_TRY(setup_batch_ingest(g.lps, count, mx, g.rp_in, g.col_in, g.val_in, g.b_in, g.sense_in,
                                g.c64, g.l64, g.u64, g.errs, s));
    ++g_launches;
    std::vector<int> errs(count);
    CUDA_TRY(cudaMemcpyAsync(errs.data(), g.errs, 4 * (size_t)count, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < count; ++k)
      if (errs[k]) {
        std::string msg = "LP " + std::to_string(k) + ": invalid input:";
        if (errs[k] & ERR_ROWPTR) msg += " row_ptr";
        if (errs[k] & ERR_COL) msg += " column index";
        if (errs[k] & ERR_NONFINITE) msg += " non-finite value";
        if (errs[k] & ERR_SENSE) msg += " sense";
        if (errs[k] & ERR_BOUNDS) msg += " bounds";
        return fail(PDLP_ERR_INVALID_INPUT, msg);
      }
  }
  // ---- A0-A3 over the whole block-diagonal problem: every step treats each row and
  // column on its own, so each LP is set up exactly as on its own
  SetupIn gin{(int)M, (int)N, Z, g.rp_in, g.col_in, g.val_in, g.b_in, g.sense_in, g.c64, g.l64, g.u64};
  CUDA_TRY(setup_canonical(gin, g.a_ptr, g.a_col, g.a_val64, g.q64, g.row_kind, s));
  CUDA_TRY(setup_transpose((int)M, (int)N, (int)Z, g.a_ptr, g.a_col, g.a_val64, g.t_ptr, g.t_col,
                           g.t_val64, g.tmp, s, false));
  g_launches += 11;
  if (p->precision == PDLP_FP32_BF16A) {
    int bf16_exact = 0, all_one = 0;
    CUDA_TRY(setup_value_format(g.a_val64, (int)Z, g.flags2, &bf16_exact, &all_one, s));
    ++g_launches;
    mode = all_one ? MODE_PAT : (bf16_exact ? MODE_BF16 : MODE_FP32);
  }
  const int scaled = (mode == MODE_FP64 || mode == MODE_FP32) ? 1 : 0;
  {
    ScaleIn sc{(int)M, (int)N, g.a_ptr, g.a_col, g.a_val64, g.t_ptr, g.t_col, g.t_val64,
               p->ruiz_iters, p->pc_alpha, Z};
    CUDA_TRY(setup_scaling(sc, g.dr, g.dc, g.stat_r, g.stat_c, s));
    g_launches += 2 + 2 * p->ruiz_iters + (p->pc_alpha >= 0 ? 2 : 0);
  }
  CUDA_TRY(setup_kkt_aux((int)M, (int)N, g.dr, g.dc, g.l64, g.u64, g.inv_dr, g.inv_dc, g.bflags, s));
  ++g_launches;
  if (mode != MODE_PAT) {
    const int vt = mode == MODE_FP64 ? 0 : (mode == MODE_FP32 ? 1 : 2);
    CUDA_TRY(setup_iter_values(vt, g.a_ptr, g.a_col, g.a_val64, (int)M, g.dr, g.dc, 1, scaled,
                               g.a_valit, s));
    CUDA_TRY(setup_iter_values(vt, g.t_ptr, g.t_col, g.t_val64, (int)N, g.dc, g.dr, 0, scaled,
                               g.t_valit, s));
    g_launches += 2;
  }
  {
    VecIn vi{(int)M, (int)N, g.dr, g.dc, g.c64, g.l64, g.u64, g.q64, g.row_kind, nullptr, nullptr,
             scaled, nullptr, nullptr};
    CUDA_TRY(setup_iter_vectors(vi, mode != MODE_FP64, g.c_it, g.l_it, g.u_it, g.q_it, g.tw, g.sw,
                                g.x[0], g.y[0], g.a_ptr, g.a_col, g.a_val64, g.part_setup,
                                g.scalars, s));
    CUDA_TRY(setup_batch_scalars(g.lps, count, g.dr, g.dc, g.c64, g.l64, g.u64, g.q64, g.a_ptr,
                                 g.a_col, g.a_val64, g.lpsca, s));
    g_launches += 4;
  }
  // long rows: one global list per orientation, each LP's part of it contiguous
  const int th_a = long_thresh(lanes[0], lanes[2]);
  const int th_t = long_thresh(lanes[1], lanes[3]);
  std::vector<int> nlong_a(count), nlong_t(count), long0_a(count), long0_t(count);
  long long la_total = 0, lt_total = 0;
  {
    int* flags = g.tmp;
    int* pos = flags + RM;
    int* bsum = pos + RM + 1;
    CUDA_TRY(setup_batch_long_rows(g.a_ptr, (int)M, th_a, g.lps, count, 0, flags, pos, bsum,
                                   g.a_long, g.lb_a, s));
    CUDA_TRY(setup_batch_long_rows(g.t_ptr, (int)N, th_t, g.lps, count, 1, flags, pos, bsum,
                                   g.t_long, g.lb_t, s));
    g_launches += 10;
    std::vector<int> lb(2 * ((size_t)count + 1));
    CUDA_TRY(cudaMemcpyAsync(lb.data(), g.lb_a, 4 * ((size_t)count + 1), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(lb.data() + count + 1, g.lb_t, 4 * ((size_t)count + 1),
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < count; ++k) {
      long0_a[k] = lb[k];
      nlong_a[k] = lb[k + 1] - lb[k];
      long0_t[k] = lb[count + 1 + k];
      nlong_t[k] = lb[count + 2 + k] - lb[count + 1 + k];
    }
    la_total = lb[count];
    lt_total = lb[2 * count + 1];
  }
  // ---- the device state of every LP (the A3 scalars of each LP)
  std::vector<double> sca(8 * (size_t)count);
  CUDA_TRY(cudaMemcpyAsync(sca.data(), g.lpsca, 8 * 8 * (size_t)count, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<DevState> hs(count);
  bool any_unboxed = false;  // some LP has a column with an infinite bound
  for (int k = 0; k < count; ++k) {
    const double* so = sca.data() + 8 * (size_t)k;
    DevState& h = hs[k];
    memset(&h, 0, sizeof(h));
    const double nct = so[0], nqt = so[1], kmax = so[4];
    h.omega = (nct > 1e-10 && nqt > 1e-10) ? nct / nqt : 1.0;
    h.eta = kmax > 0.0 ? 1.0 / kmax : 1.0;
    if (p->fixed_eta > 0.0) h.eta = p->fixed_eta;
    if (p->fixed_omega > 0.0) h.omega = p->fixed_omega;
    h.check_due = 1;
    h.init_pending = 1;
    h.prev_cand = INFINITY;
    h.iter_limit = p->iter_limit;
    h.period = p->check_period;
    h.adaptive = p->adaptive_step ? 1 : 0;
    h.restarts_on = p->restarts ? 1 : 0;
    h.terminate = p->terminate ? 1 : 0;
    h.detect_inf = p->detect_infeasibility ? 1 : 0;
    h.spin_limit = kSpinLimit;
    h.tol = p->tol;
    h.norm_c = so[2];
    h.norm_q = so[3];
    any_unboxed = any_unboxed || so[7] > 0.0;
    h.inv_omega = 1.0 / h.omega;
    h.tau_d = h.eta / h.omega;
    h.sigma_d = h.eta * h.omega;
    h.eta_f = (float)h.eta;
    h.omega_f = (float)h.omega;
    h.inv_omega_f = (float)h.inv_omega;
    h.tau_f = h.eta_f * h.inv_omega_f;
    h.sigma_f = h.eta_f * h.omega_f;
    h.fac_dec = g.fac->dec;
    h.fac_inc = g.fac->inc;
    h.fac_dec_f = g.fac->dec_f;
    h.fac_inc_f = g.fac->inc_f;
    h.fac_n = kFacN;
  }
  {
    CUDA_TRY(cudaMemsetAsync(g.sum_x, 0, eb * N, s));
    if (M) CUDA_TRY(cudaMemsetAsync(g.sum_y, 0, eb * M, s));
    CUDA_TRY(cudaMemsetAsync(g.Xl, 0, 8 * N, s));
    if (M) CUDA_TRY(cudaMemsetAsync(g.Yl, 0, 8 * M, s));
    CUDA_TRY(cudaMemcpyAsync(g.st, hs.data(), sizeof(DevState) * count, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  // ---- launch maps
  const bool tiled = mode == MODE_FP64;
  std::vector<int> tabA, tabT;
  int gridA = 0, gridT = 0;
  build_map(sh, false, lanes[0], tiled, nlong_a, long0_a, M, budget, tabA, &gridA);
  build_map(sh, true, lanes[1], tiled, nlong_t, long0_t, N, budget, tabT, &gridT);
  if ((size_t)gridA > gmax || (size_t)gridT > gmax) return fail(PDLP_ERR_OOM, "launch map too large");
  CUDA_TRY(cudaMemcpyAsync(g.tabA, tabA.data(), 4 * tabA.size(), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(g.tabT, tabT.data(), 4 * tabT.size(), cudaMemcpyHostToDevice, s));
  const Tables tA = tables_at(g.tabA, gridA, count), tT = tables_at(g.tabT, gridT, count);
  IterRaw ir{};
  ir.a_ptr = g.a_ptr; ir.a_col = g.a_col; ir.a_val = mode == MODE_PAT ? nullptr : g.a_valit;
  ir.t_ptr = g.t_ptr; ir.t_col = g.t_col; ir.t_val = mode == MODE_PAT ? nullptr : g.t_valit;
  ir.a_long = g.a_long; ir.t_long = g.t_long;
  ir.a_nlong = (int)la_total; ir.t_nlong = (int)lt_total; ir.a_thresh = th_a; ir.t_thresh = th_t;
  ir.m = (int)M; ir.n = (int)N;
  ir.c = g.c_it; ir.l = g.l_it; ir.u = g.u_it; ir.q = g.q_it;
  ir.tw = scaled ? nullptr : g.tw; ir.sw = scaled ? nullptr : g.sw;
  ir.row_kind = g.row_kind;
  for (int k = 0; k < 2; ++k) { ir.x[k] = g.x[k]; ir.y[k] = g.y[k]; }
  ir.sum_x = g.sum_x; ir.sum_y = g.sum_y;
  ir.part_p = g.part_p; ir.part_d = g.part_d;
  ir.grid_p_short = gridT; ir.grid_p = gridT; ir.grid_d_short = gridA; ir.grid_d = gridA;
  ir.st = g.st;
  ir.count = count;
  ir.tp = tT;
  ir.td = tA;
  if (use_tiles) {
    // work items over the global A and A^T, none straddling two LPs
    std::vector<int> r0a(count + 1), r0t(count + 1);
    for (int k = 0; k < count; ++k) {
      r0a[k] = (int)sh[k].R;
      r0t[k] = (int)sh[k].C;
    }
    r0a[count] = (int)M;
    r0t[count] = (int)N;
    CUDA_TRY(cudaMemcpyAsync(g.row0_a, r0a.data(), 4 * (count + 1), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(g.row0_t, r0t.data(), 4 * (count + 1), cudaMemcpyHostToDevice, s));
    int ca[2] = {0, 0}, ct[2] = {0, 0}, W = 0;
    CUDA_TRY(setup_tiles(tsh, g.a_ptr, (int)M, Z, g.row0_a, count, g.tmp, g.ti_a, g.tlp_a,
                         g.tlp_a + count + 1, g.tick_a, tcap_a, ca, &W, s));
    CUDA_TRY(setup_tiles(tsh, g.t_ptr, (int)N, Z, g.row0_t, count, g.tmp, g.ti_t, g.tlp_t,
                         g.tlp_t + count + 1, g.tick_t, tcap_t, ct, &W, s));
    g_launches += 16;
    int bp = 0, bd = 0;
    CUDA_TRY(tile_resident_mode((Mode)mode, p->tiles, &bp, &bd));
    ir.tile = p->tiles;
    ir.tslot = (int)tslot;
    ir.tt = TileSet{g.ti_t, ct[0], g.tlp_t, g.tlp_t + count + 1, g.tpart_t, g.trow_t, g.tlong_t, g.tick_t};
    ir.ta = TileSet{g.ti_a, ca[0], g.tlp_a, g.tlp_a + count + 1, g.tpart_a, g.trow_a, g.tlong_a, g.tick_a};
    tile_launch(p->tiles, ct[0], bp, &ir.grid_tt, &ir.work_tt);
    tile_launch(p->tiles, ca[0], bd, &ir.grid_ta, &ir.work_ta);
  }
  KktRaw kr{};
  kr.a_ptr = g.a_ptr; kr.a_col = g.a_col; kr.a_val64 = mode == MODE_PAT ? nullptr : g.a_val64;
  kr.t_ptr = g.t_ptr; kr.t_col = g.t_col; kr.t_val64 = mode == MODE_PAT ? nullptr : g.t_val64;
  kr.a_long = g.a_long; kr.t_long = g.t_long;
  kr.a_nlong = (int)la_total; kr.t_nlong = (int)lt_total; kr.a_thresh = th_a; kr.t_thresh = th_t;
  kr.m = (int)M; kr.n = (int)N;
  kr.c = g.c64; kr.l = g.l64; kr.u = g.u64; kr.q = g.q64; kr.dr = g.dr; kr.dc = g.dc;
  kr.inv_dr = g.inv_dr; kr.inv_dc = g.inv_dc; kr.bflags = g.bflags;
  kr.row_kind = g.row_kind;
  for (int k = 0; k < 2; ++k) { kr.x[k] = g.x[k]; kr.y[k] = g.y[k]; }
  kr.sum_x = g.sum_x; kr.sum_y = g.sum_y;
  kr.XG = g.XG; kr.Xl = g.Xl; kr.YG = g.YG; kr.Yl = g.Yl; kr.XR = g.XR; kr.YR = g.YR;
  kr.rays = p->detect_infeasibility && p->terminate ? (any_unboxed ? 2 : 1) : 0;
  kr.part_r = g.part_r; kr.part_c = g.part_c;
  kr.grid_r_short = gridA; kr.grid_r = gridA; kr.grid_c_short = gridT; kr.grid_c = gridT;
  kr.grid_e = gridT;
  kr.scaled = scaled; kr.fp32 = mode != MODE_FP64;
  kr.ux = kr.uy = 1.0;  // batches: no bound-objective rescaling
  kr.st = g.st;
  kr.count = count;
  kr.tr = tA;
  kr.tc = tT;
  Solve sv{(int)M, (int)N, Z, (Mode)mode, lanes[0], lanes[1], lanes[2], lanes[3], ir, kr, s, 0};
  if (p->autotune && !use_tiles && (!p->lanes_A || !p->lanes_AT) && p->iter_limit > 0) {
    // a lanes choice changes the blocks each LP gets: rebuild both launch maps
    auto set_grids = [&](int lt, int la) -> int {
      build_map(sh, false, la, tiled, nlong_a, long0_a, M, budget, tabA, &gridA);
      build_map(sh, true, lt, tiled, nlong_t, long0_t, N, budget, tabT, &gridT);
      if ((size_t)gridA > gmax || (size_t)gridT > gmax) return fail(PDLP_ERR_OOM, "launch map too large");
      CUDA_TRY(cudaMemcpyAsync(g.tabA, tabA.data(), 4 * tabA.size(), cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaMemcpyAsync(g.tabT, tabT.data(), 4 * tabT.size(), cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors are refilled next time
      const Tables a2 = tables_at(g.tabA, gridA, count), t2 = tables_at(g.tabT, gridT, count);
      sv.ir.grid_p_short = sv.ir.grid_p = gridT;
      sv.ir.grid_d_short = sv.ir.grid_d = gridA;
      sv.ir.tp = t2;
      sv.ir.td = a2;
      sv.kr.grid_r_short = sv.kr.grid_r = gridA;
      sv.kr.grid_c_short = sv.kr.grid_c = gridT;
      sv.kr.grid_e = gridT;
      sv.kr.tr = a2;
      sv.kr.tc = t2;
      return PDLP_OK;
    };
    std::vector<DevState> hst(count);
    auto set_dry = [&](bool on) -> int {
      CUDA_TRY(cudaMemcpyAsync(hst.data(), g.st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      for (DevState& h : hst) {
        h.check_due = on ? 0 : 1;
        h.dry = on ? 1 : 0;
      }
      CUDA_TRY(cudaMemcpyAsync(g.st, hst.data(), sizeof(DevState) * count, cudaMemcpyHostToDevice, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      return PDLP_OK;
    };
    const int rc = autotune_lanes(sv, count, !p->lanes_AT, !p->lanes_A, one_ok, set_grids,
                                  set_dry);
    if (rc) return rc;
    lanes[0] = sv.lanes_a;
    lanes[1] = sv.lanes_t;
    ir = sv.ir;  // the output kernels below use these copies
    kr = sv.kr;
  }
  if (p->persistent == 1) {
    // one cooperative kernel per check period walks both launch maps with the resident
    // grid (probe launch with no attempt to run: the states say check_due)
    int gp = 0;
    cudaError_t e;
    switch (mode) {
      case MODE_FP64: e = launch_persist_fp64(sv.lanes_a, sv.lanes_t, sv.ir, 0, 0, &gp, s); break;
      case MODE_FP32: e = launch_persist_fp32(sv.lanes_a, sv.lanes_t, sv.ir, 0, 0, &gp, s); break;
      case MODE_BF16: e = launch_persist_bf16(sv.lanes_a, sv.lanes_t, sv.ir, 0, 0, &gp, s); break;
      default: e = launch_persist_pat(sv.lanes_a, sv.lanes_t, sv.ir, 0, 0, &gp, s); break;
    }
    ++g_launches;
    if (e != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("persistent kernel: ") + cudaGetErrorString(e));
    sv.persist_grid = gp;
  }
  CUDA_TRY(sv.kkt_block());  // initial KKT of every LP
  CUDA_TRY(cudaStreamSynchronize(s));
  if (tq) return time_kernels_after_setup(sv, g.st, mode, Z, *tq, count);
  const double setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // ---- iteration phase: one graph of a check period for the whole batch
  const auto t1 = std::chrono::steady_clock::now();
  if (p->iter_limit > 0) {
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    Solve cap = sv;
    cap.s = cs;
    Fork fork;
    {
      const cudaError_t fe = fork.make(cap);
      if (fe != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(PDLP_ERR_CUDA, std::string("fork stream: ") + cudaGetErrorString(fe));
      }
    }
    const long long before = g_launches;
    cudaGraph_t graph;
    CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cap.period_steps(p->check_period);
    if (ce == cudaSuccess) ce = cap.kkt_block();
    cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) return fail(PDLP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    CUDA_TRY(ee);
    const long long nodes = g_launches - before;
    g_launches = before;
    cudaGraphExec_t ge;
    cudaError_t ie = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(ie);
    struct GFree {
      cudaGraphExec_t g;
      ~GFree() { cudaGraphExecDestroy(g); }
    } gfree{ge};
    DevState* hm = nullptr;
    CUDA_TRY(cudaMallocHost(&hm, sizeof(DevState) * count));
    struct HFree {
      void* p;
      ~HFree() { cudaFreeHost(p); }
    } hfree{hm};
    const long long max_launches = (p->iter_limit / p->check_period + 2) * 64 + 1024;
    bool forced = false;
    static const int one_flag[2] = {1, 1};
    for (long long launch = 0;; ++launch) {
      CUDA_TRY(cudaGraphLaunch(ge, s));
      g_launches += nodes;
      CUDA_TRY(cudaMemcpyAsync(hm, g.st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(cudaStreamSynchronize(s));
      int running = 0;
      for (int k = 0; k < count; ++k) running += hm[k].status == 0;
      if (!running) break;
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
      if (!forced && el > p->time_limit_s) {
        for (int k = 0; k < count; ++k) {
          CUDA_TRY(cudaMemcpyAsync(&g.st[k].force_final, &one_flag[0], sizeof(int), cudaMemcpyHostToDevice, s));
          CUDA_TRY(cudaMemcpyAsync(&g.st[k].check_due, &one_flag[1], sizeof(int), cudaMemcpyHostToDevice, s));
        }
        forced = true;
      }
      if (launch > max_launches) return fail(PDLP_ERR_TIMEOUT, "batch iteration loop did not terminate");
    }
  }
  const double solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
  {
    std::vector<DevState> chk(count);
    CUDA_TRY(cudaMemcpyAsync(chk.data(), g.st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (const DevState& f : chk)
      if (f.status == kStatusWaitFailed)
        return fail(PDLP_ERR_TIMEOUT, "a bounded wait of a step kernel gave up");
  }
  // ---- outputs
  CUDA_TRY(launch_output(kr, g.x_out, M ? g.y_out : nullptr, nullptr, nullptr, nullptr, nullptr, s));
  ++g_launches;
  std::vector<DevState> fs(count);
  CUDA_TRY(cudaMemcpyAsync(fs.data(), g.st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
  for (int k = 0; k < count; ++k) {
    const cudaMemcpyKind kind = device_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x_out && x_out[k])
      CUDA_TRY(cudaMemcpyAsync(x_out[k], g.x_out + sh[k].C, 8 * (size_t)sh[k].n, kind, s));
    if (y_out && y_out[k] && sh[k].m)
      CUDA_TRY(cudaMemcpyAsync(y_out[k], g.y_out + sh[k].R, 8 * (size_t)sh[k].m, kind, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < count; ++k) {
    pdlp_result& r = res[k];
    memset(&r, 0, sizeof(r));
    const DevState& f = fs[k];
    r.status = p->iter_limit == 0 ? PDLP_ITER_LIMIT : f.status;
    r.precision_used = mode == MODE_FP64 ? PDLP_FP64 : mode == MODE_FP32 ? PDLP_FP32
                       : mode == MODE_BF16 ? PDLP_USED_BF16 : PDLP_USED_PATTERN;
    r.lanes_A = lanes[0];
    r.lanes_AT = lanes[1];
    r.tiles = ir.tile;
    r.persistent_form = sv.persist_grid > 0 ? 1 : 0;
    r.iters = f.iters;
    r.attempts = f.attempts;
    r.restarts = f.restarts;
    r.kkt_checks = f.checks;
    const int a = f.used_avg ? 1 : 0;
    r.used_average = a;
    r.primal_obj = f.pobj[a];
    r.dual_obj = f.dobj[a];
    r.rel_primal_res = f.relp[a];
    r.rel_dual_res = f.reld[a];
    r.rel_gap = f.relgap[a];
    r.rel_kkt = std::max(r.rel_primal_res, std::max(r.rel_dual_res, r.rel_gap));
    r.eta = f.eta;
    r.omega = f.omega;
    const bool cert = f.status == PDLP_PRIMAL_INFEASIBLE || f.status == PDLP_DUAL_INFEASIBLE;
    r.ray_obj = cert ? f.ray_obj : NAN;
    r.ray_res = cert ? f.ray_res : NAN;
    r.setup_s = setup_s - upload_s;
    r.upload_s = upload_s;
    r.solve_s = solve_s;
    r.kernel_launches = g_launches;
  }
  return PDLP_OK;
}

int set_error(int code, const char* msg) { return fail(code, msg); }

// pdlp_solve_device on caller-provided scratch without creating any CUDA
// object or allocating (see noalloc.cu)
int solve_device_noalloc(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                         const double* l, const double* u, const pdlp_params* p, const double* x0,
                         const double* y0, double* x_out, double* y_out, pdlp_result* r,
                         const pdlp_diagnostics* dg, void* workspace, size_t ws_bytes,
                         cudaStream_t s) {
  const int rc = check_inputs(A, b, sense, c, l, u, p, x_out, y_out, r);
  if (rc) return rc;
  return solve_device(A, b, sense, c, l, u, p, x0, y0, x_out, y_out, r, dg, workspace, ws_bytes,
                      s, nullptr, true);
}

}  // namespace pdlp

using namespace pdlp;

extern "C" {

int pdlp_default_params(pdlp_params* p) {
  if (!p) return fail(PDLP_ERR_INVALID_INPUT, "NULL params");
  memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(pdlp_params);
  p->tol = 1e-4;
  p->iter_limit = 1000000;
  p->time_limit_s = 3600.0;
  p->precision = PDLP_FP64;
  p->check_period = 64;
  p->ruiz_iters = 10;
  p->pc_alpha = 1.0;
  p->adaptive_step = 1;
  p->restarts = 1;
  p->terminate = 1;
  p->persistent = 0;
  p->autotune = 0;
  p->detect_infeasibility = 1;
  p->tiles = 0;
  p->bound_objective_rescaling = 0;
  p->halpern = 0;
  p->halpern_reflection = 1.0;
  p->restart_metric = 0;
  return PDLP_OK;
}

size_t pdlp_workspace_size(int32_t m, int32_t n, int64_t nnz, const pdlp_params* p) {
  if (m < 0 || n < 1 || nnz < 0 || nnz >= (int64_t)INT32_MAX) return 0;
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  Bufs b;
  Arena ar{nullptr, 0};
  return carve(ar, b, m, n, nnz, p->precision, p->restart_metric == 1);
}

int pdlp_solve_device(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, double* x_out, double* y_out, pdlp_result* r,
                      const pdlp_diagnostics* diag, void* workspace, size_t workspace_bytes,
                      void* stream) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  int rc = check_inputs(A, b, sense, c, l, u, p, x_out, y_out, r);
  if (rc) return rc;
  return solve_device(A, b, sense, c, l, u, p, x0, y0, x_out, y_out, r, diag, workspace,
                      workspace_bytes, (cudaStream_t)stream);
}

}  // extern "C"

namespace pdlp {

// pdlp_solve and pdlp_solve_hinted: host buffers in, one device block for the
// inputs, outputs, diagnostics and workspace
static int solve_host(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, const double* hx, const double* hy, double* x_out,
                      double* y_out, pdlp_result* r, const pdlp_diagnostics* diag) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  int rc = check_inputs(A, b, sense, c, l, u, p, x_out, y_out, r);
  if (rc) return rc;
  const size_t M = (size_t)A->m, N = (size_t)A->n, Z = (size_t)A->nnz;
  const size_t TA = diag && diag->attempt_capacity > 0 ? (size_t)diag->attempt_capacity : 0;
  const size_t TC = diag && diag->check_capacity > 0 ? (size_t)diag->check_capacity : 0;
  const size_t TP = diag && diag->point_capacity > 0 && diag->check_points
                        ? (size_t)diag->point_capacity : 0;
  cudaStream_t s;
  CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  struct StreamFree {
    cudaStream_t s;
    ~StreamFree() { cudaStreamDestroy(s); }
  } sfree{s};
  // one device block for the inputs, outputs and diagnostics
  auto lay = [&](Arena& ar, void** ptrs) {
    ptrs[0] = ar.take(8 * (M + 1));  // row_ptr
    ptrs[1] = ar.take(4 * Z);        // col
    ptrs[2] = ar.take(8 * Z);        // val
    ptrs[3] = ar.take(8 * M);        // b
    ptrs[4] = ar.take(M);            // sense
    ptrs[5] = ar.take(8 * N);        // c
    ptrs[6] = ar.take(8 * N);        // l
    ptrs[7] = ar.take(8 * N);        // u
    ptrs[8] = ar.take(8 * N);        // x0
    ptrs[9] = ar.take(8 * M);        // y0
    ptrs[10] = ar.take(8 * N);       // x_out
    ptrs[11] = ar.take(8 * M);       // y_out
    for (int k = 0; k < 4; ++k) ptrs[12 + k] = ar.take(8 * ((k & 1) ? M : N));  // iterates
    ptrs[16] = ar.take(8 * TA);      // eta
    ptrs[17] = ar.take(8 * TA);      // eta_bar
    ptrs[18] = ar.take(TA);          // accepted
    ptrs[19] = ar.take(TC);          // restart
    ptrs[20] = ar.take(8 * TC);      // omega
    ptrs[21] = ar.take(8 * N);       // primal-weight hint x
    ptrs[22] = ar.take(8 * M);       // primal-weight hint y
    ptrs[23] = ar.take(8 * TP * N);  // check points
  };
  void* dp[24];
  Arena dry{nullptr, 0};
  lay(dry, dp);
  const size_t io_bytes = dry.off + 256;
  const size_t ws_bytes = pdlp_workspace_size(A->m, A->n, A->nnz, p);
  void* dev = nullptr;
  {
    cudaError_t e = cudaMallocAsync(&dev, io_bytes + ws_bytes + 256, s);
    if (e != cudaSuccess) return fail(PDLP_ERR_OOM, std::string("device buffers: ") + cudaGetErrorString(e));
  }
  struct DevFree {
    void* p;
    cudaStream_t s;
    ~DevFree() {
      cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } dfree{dev, s};
  Arena ar{(char*)dev, 0};
  lay(ar, dp);
  void* ws = (char*)dev + ((io_bytes + 255) & ~(size_t)255);
  auto h2d = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    return bytes && src ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  auto d2h = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    return bytes && dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
  };
  CUDA_TRY(h2d(dp[0], A->row_ptr, 8 * (M + 1)));
  CUDA_TRY(h2d(dp[1], A->col, 4 * Z));
  CUDA_TRY(h2d(dp[2], A->val, 8 * Z));
  CUDA_TRY(h2d(dp[3], b, 8 * M));
  CUDA_TRY(h2d(dp[4], sense, M));
  CUDA_TRY(h2d(dp[5], c, 8 * N));
  CUDA_TRY(h2d(dp[6], l, 8 * N));
  CUDA_TRY(h2d(dp[7], u, 8 * N));
  CUDA_TRY(h2d(dp[8], x0, 8 * N));
  CUDA_TRY(h2d(dp[9], y0, 8 * M));
  CUDA_TRY(h2d(dp[21], hx, 8 * N));
  CUDA_TRY(h2d(dp[22], hy, 8 * M));
  pdlp_csr dA{A->m, A->n, A->nnz, (const int64_t*)dp[0], (const int32_t*)dp[1], (const double*)dp[2]};
  pdlp_diagnostics ddg{(double*)dp[12], (double*)dp[13], (double*)dp[14], (double*)dp[15],
                       (int64_t)TA, (double*)dp[16], (double*)dp[17], (int8_t*)dp[18],
                       (int64_t)TC, (int8_t*)dp[19], (double*)dp[20], (int64_t)TP,
                       TP ? (double*)dp[23] : nullptr};
  rc = solve_device(&dA, (const double*)dp[3], (const char*)dp[4], (const double*)dp[5],
                    (const double*)dp[6], (const double*)dp[7], p, x0 ? (const double*)dp[8] : nullptr,
                    y0 ? (const double*)dp[9] : nullptr, (double*)dp[10], (double*)dp[11], r,
                    diag ? &ddg : nullptr, ws, ws_bytes, s, nullptr, false,
                    hx ? (const double*)dp[21] : nullptr, hy ? (const double*)dp[22] : nullptr);
  if (rc) return rc;
  CUDA_TRY(d2h(x_out, dp[10], 8 * N));
  CUDA_TRY(d2h(y_out, dp[11], 8 * M));
  if (diag) {
    CUDA_TRY(d2h(diag->x_cur, dp[12], 8 * N));
    CUDA_TRY(d2h(diag->y_cur, dp[13], 8 * M));
    CUDA_TRY(d2h(diag->x_avg, dp[14], 8 * N));
    CUDA_TRY(d2h(diag->y_avg, dp[15], 8 * M));
    if (diag->eta && diag->eta_bar && diag->accepted) {
      CUDA_TRY(d2h(diag->eta, dp[16], 8 * TA));
      CUDA_TRY(d2h(diag->eta_bar, dp[17], 8 * TA));
      CUDA_TRY(d2h(diag->accepted, dp[18], TA));
    }
    if (diag->restart && diag->omega) {
      CUDA_TRY(d2h(diag->restart, dp[19], TC));
      CUDA_TRY(d2h(diag->omega, dp[20], 8 * TC));
    }
    if (TP) CUDA_TRY(d2h(diag->check_points, dp[23], 8 * TP * N));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return PDLP_OK;
}

// pdlp_solve_device with a primal-weight hint (device buffers), used by the
// learned warm start
int solve_device_hint(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, const double* hx, const double* hy, double* x_out,
                      double* y_out, pdlp_result* r, cudaStream_t s) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  const int rc = check_inputs(A, b, sense, c, l, u, p, x_out, y_out, r);
  if (rc) return rc;
  return solve_device(A, b, sense, c, l, u, p, x0, y0, x_out, y_out, r, nullptr, nullptr, 0, s,
                      nullptr, false, hx, hy);
}

}  // namespace pdlp

extern "C" {

int pdlp_solve(const pdlp_csr* A, const double* b, const char* sense, const double* c,
               const double* l, const double* u, const pdlp_params* p, const double* x0,
               const double* y0, double* x_out, double* y_out, pdlp_result* r,
               const pdlp_diagnostics* diag) {
  return solve_host(A, b, sense, c, l, u, p, x0, y0, nullptr, nullptr, x_out, y_out, r, diag);
}

int pdlp_solve_hinted(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, const double* x_hint, const double* y_hint,
                      double* x_out, double* y_out, pdlp_result* r,
                      const pdlp_diagnostics* diag) {
  if (!x_hint || (!y_hint && A && A->m > 0))
    return fail(PDLP_ERR_INVALID_INPUT, "pdlp_solve_hinted needs x_hint[n] and y_hint[m]");
  return solve_host(A, b, sense, c, l, u, p, x0, y0, x_hint, y_hint, x_out, y_out, r, diag);
}

int pdlp_polish_primal(const pdlp_csr* A, const double* b, const char* sense, const double* l,
                       const double* u, const pdlp_params* p, const double* x_in,
                       double* x_out, double* y_out, pdlp_result* r) {
  if (!A || A->n < 1 || !x_in || !x_out)
    return fail(PDLP_ERR_INVALID_INPUT, "pdlp_polish_primal needs A, x_in[n] and x_out[n]");
  // the objective-free problem from (x_in, 0)
  const std::vector<double> zero_c((size_t)A->n, 0.0);
  std::vector<double> y_tmp;
  if (!y_out && A->m > 0) {
    y_tmp.resize((size_t)A->m);
    y_out = y_tmp.data();
  }
  return solve_host(A, b, sense, zero_c.data(), l, u, p, x_in, nullptr, nullptr, nullptr, x_out,
                    y_out, r, nullptr);
}

int pdlp_polish_dual(const pdlp_csr* A, const char* sense, const double* c, const double* l,
                     const double* u, const pdlp_params* p, const double* y_in, double* x_out,
                     double* y_out, pdlp_result* r) {
  if (!A || A->n < 1 || A->m < 0 || (A->m > 0 && (!y_in || !y_out)) || !c || !l || !u)
    return fail(PDLP_ERR_INVALID_INPUT, "pdlp_polish_dual needs A, c, l, u, y_in[m] and y_out[m]");
  // the dual feasibility problem from (0, y_in): b = 0, finite bounds moved to 0
  const size_t N = (size_t)A->n;
  const std::vector<double> zero_b((size_t)A->m, 0.0);
  std::vector<double> l0(N), u0(N), x_tmp;
  for (size_t j = 0; j < N; ++j) {
    if (l[j] > u[j]) return fail(PDLP_ERR_INVALID_INPUT, "l > u in column " + std::to_string(j));
    l0[j] = std::isfinite(l[j]) ? 0.0 : l[j];  // NaN stays NaN: the setup rejects it
    u0[j] = std::isfinite(u[j]) ? 0.0 : u[j];
  }
  if (!x_out) {
    x_tmp.resize(N);
    x_out = x_tmp.data();
  }
  return solve_host(A, zero_b.data(), sense, c, l0.data(), u0.data(), p, nullptr, y_in, nullptr,
                    nullptr, x_out, y_out, r, nullptr);
}

int pdlp_time_kernels(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, int reps,
                      double* ms_per_launch, double* bytes_per_launch, void* workspace,
                      size_t workspace_bytes, void* stream) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  if (reps < 1 || !ms_per_launch || !bytes_per_launch)
    return fail(PDLP_ERR_INVALID_INPUT, "reps >= 1 and output arrays required");
  double xo = 0.0;
  int rc = check_inputs(A, b, sense, c, l, u, p, &xo, &xo, (const pdlp_result*)&xo);
  if (rc) return rc;
  pdlp_result r;
  TimingReq tq{reps, ms_per_launch, bytes_per_launch};
  return solve_device(A, b, sense, c, l, u, p, nullptr, nullptr, nullptr, nullptr, &r, nullptr,
                      workspace, workspace_bytes, (cudaStream_t)stream, &tq);
}

int pdlp_solve_batch(int count, const pdlp_csr* const* A, const double* const* b,
                     const char* const* sense, const double* const* c, const double* const* l,
                     const double* const* u, const pdlp_params* p, double* const* x_out,
                     double* const* y_out, pdlp_result* r) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  if (count < 1 || !A || !b || !sense || !c || !l || !u || !r)
    return fail(PDLP_ERR_INVALID_INPUT, "batch: count >= 1 and every pointer array required");
  for (int k = 0; k < count; ++k) {
    double dummy = 0.0;
    const int rc = check_inputs(A[k], b[k], sense[k], c[k], l[k], u[k], p,
                                x_out ? (void*)x_out[k] : (void*)&dummy,
                                (y_out && y_out[k]) ? (void*)y_out[k] : (void*)&dummy, &r[k]);
    if (rc) return fail(rc, std::string("LP ") + std::to_string(k) + ": " + g_last_error);
  }
  return solve_batch(count, A, b, sense, c, l, u, p, x_out, y_out, r);
}

int pdlp_solve_batch_device(int count, const pdlp_csr* const* A, const double* const* b,
                            const char* const* sense, const double* const* c,
                            const double* const* l, const double* const* u, const pdlp_params* p,
                            double* const* x_out, double* const* y_out, pdlp_result* r,
                            void* stream) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  if (count < 1 || !A || !b || !sense || !c || !l || !u || !r)
    return fail(PDLP_ERR_INVALID_INPUT, "batch: count >= 1 and every pointer array required");
  for (int k = 0; k < count; ++k) {
    double dummy = 0.0;
    const int rc = check_inputs(A[k], b[k], sense[k], c[k], l[k], u[k], p,
                                x_out ? (void*)x_out[k] : (void*)&dummy,
                                (y_out && y_out[k]) ? (void*)y_out[k] : (void*)&dummy, &r[k]);
    if (rc) return fail(rc, std::string("LP ") + std::to_string(k) + ": " + g_last_error);
  }
  return solve_batch(count, A, b, sense, c, l, u, p, x_out, y_out, r, nullptr, true,
                     (cudaStream_t)stream);
}

int pdlp_time_kernels_batch(int count, const pdlp_csr* const* A, const double* const* b,
                            const char* const* sense, const double* const* c,
                            const double* const* l, const double* const* u, const pdlp_params* p,
                            int reps, double* ms_per_launch, double* bytes_per_launch) {
  pdlp_params d;
  if (!p) {
    pdlp_default_params(&d);
    p = &d;
  }
  if (count < 1 || !A || !b || !sense || !c || !l || !u || reps < 1 || !ms_per_launch ||
      !bytes_per_launch)
    return fail(PDLP_ERR_INVALID_INPUT, "batch timing: count >= 1, reps >= 1 and every array required");
  std::vector<pdlp_result> r((size_t)count);
  for (int k = 0; k < count; ++k) {
    double dummy = 0.0;
    const int rc = check_inputs(A[k], b[k], sense[k], c[k], l[k], u[k], p, &dummy, &dummy, &r[k]);
    if (rc) return fail(rc, std::string("LP ") + std::to_string(k) + ": " + g_last_error);
  }
  TimingReq tq{reps, ms_per_launch, bytes_per_launch};
  return solve_batch(count, A, b, sense, c, l, u, p, nullptr, nullptr, r.data(), &tq);
}

const char* pdlp_error_string(int code) {
  switch (code) {
    case PDLP_OK: return "PDLP_OK";
    case PDLP_ERR_INVALID_INPUT: return "PDLP_ERR_INVALID_INPUT";
    case PDLP_ERR_CUDA: return "PDLP_ERR_CUDA";
    case PDLP_ERR_OOM: return "PDLP_ERR_OOM";
    case PDLP_ERR_TIMEOUT: return "PDLP_ERR_TIMEOUT";
    case PDLP_ERR_UNSUPPORTED: return "PDLP_ERR_UNSUPPORTED";
    default: return "PDLP_ERR_UNKNOWN";
  }
}

const char* pdlp_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
