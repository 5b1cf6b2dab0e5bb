// Shared device-side definitions of the PDLP library: the device-resident
// solver state, value loaders for the matrix storage formats, and the
// deterministic warp / block reductions every fused kernel ends with.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace pdlp {

constexpr int kBlock = 256;         // threads per block of every streaming kernel
constexpr int kWarps = kBlock / 32;
// resident blocks per SM the float32 step kernels are compiled for
constexpr int kStepBlocksPerSmF32 = 4;
// static shared memory the one-block shared-memory step kernel keeps for itself (its
// copy of the state and the block reductions), subtracted from the device's opt-in limit
constexpr int kSmemStatic = 8192;

// Matrix value formats of the iteration matrix.
struct Pattern {};  // every stored value is exactly +1: no value array at all

template <typename V> __device__ __forceinline__ float ldv_f(const V* v, int64_t p);
template <> __device__ __forceinline__ float ldv_f<float>(const float* v, int64_t p) { return __ldg(v + p); }
template <> __device__ __forceinline__ float ldv_f<__nv_bfloat16>(const __nv_bfloat16* v, int64_t p) {
  return __bfloat162float(v[p]);
}
template <> __device__ __forceinline__ float ldv_f<Pattern>(const Pattern*, int64_t) { return 1.0f; }

template <typename T, typename V> struct Ld;
template <typename V> struct Ld<float, V> {
  static __device__ __forceinline__ float get(const V* v, int64_t p) { return ldv_f<V>(v, p); }
};
template <> struct Ld<double, double> {
  static __device__ __forceinline__ double get(const double* v, int64_t p) { return __ldg(v + p); }
};

// Device-resident solver state.  Written by one thread of the deciding block
// (the step-decision kernel, the KKT finalisation kernel) and
// read by every kernel at entry; kernels launched after a terminating or a
// KKT-pending decision return immediately, so a captured chunk of iterations
// is safe to over-launch.
struct DevState {
  // host-visible summary first (copied back after every chunk)
  int status;            // 0 running, else PDLP_OPTIMAL / ITER_LIMIT / TIME_LIMIT / NUMERICAL /
                         // PRIMAL_INFEASIBLE / DUAL_INFEASIBLE
  int check_due;         // 1: the KKT block must run before the next step
  long long iters;       // accepted iterations
  long long attempts;    // all step attempts (k of the step-size rule, 1-based after increment)
  long long restarts;
  long long checks;
  // step size / primal weight (A3, A6, A10)
  double eta, omega;
  // weighted averages (A7): sum_w includes pending_w; the iterate whose weight
  // is pending has not yet been added to sum_x / sum_y (the next step adds it
  // while it reads that iterate anyway)
  double sum_w, pending_w;
  int cur;               // which of the two x / y buffers holds the current iterate
  int restart_kind;      // set by the KKT finalisation: 0 none, 1 to current, 2 to average, 3 initial
  int init_pending;      // the first KKT block only records the "last restart" data
  int used_avg;          // output candidate of the last check
  int force_final;       // host asked for a final check (time limit)
  int dry;               // 1: step kernels run but the decision is skipped (launch-shape tuning)
  int loop_attempts;     // attempts since the start of the current check-period graph
  long long last_restart_it;
  double last_rp2, last_rd2, last_gap2;  // scaled KKT triple of the last restart point
  double prev_cand;                      // KKT_omega of the previous candidate (inf after restart)
  // parameters
  long long iter_limit;
  int period, adaptive, restarts_on, terminate;
  int detect_inf;         // 1: test the certificates of infeasibility at each check
  double tol;
  // certificate of the terminating check (status 5 / 6): its ray objective and
  // the norm of its residual
  double ray_obj, ray_res;
  double norm_q, norm_c;  // ||q||_2, ||c||_2 of the unscaled data
  // results of the last KKT check: [0] current, [1] average
  double pobj[2], dobj[2], relp[2], reld[2], relgap[2];
  // per-attempt scalars prepared by the deciding thread, in both precisions, so
  // the step kernels run no float64 arithmetic in the float32 modes:
  //   tau = eta / omega, sigma = eta * omega, pw = pending_w
  double tau_d, sigma_d, inv_omega;
  float tau_f, sigma_f, pw_f, eta_f, omega_f, inv_omega_f;
  // step-rule factors 1 - (k+1)^-0.3 and 1 + (k+1)^-0.6 for attempts k = 1..fac_n
  // (computed on the host with the C library pow; beyond the table, pow here)
  const double* fac_dec;
  const double* fac_inc;
  const float* fac_dec_f;
  const float* fac_inc_f;
  long long fac_n;
  // optional decision trace (device arrays, capacity 0 = off)
  double* tr_eta;
  double* tr_eta_bar;
  signed char* tr_accepted;
  long long tr_cap;
  signed char* tr_restart;
  double* tr_omega;
  long long tr_check_cap;
  // grid barrier of the persistent step kernel (arrivals, generation, failure flag)
  unsigned int bar_count, bar_gen;
  int bar_err;
  int bar_skip;          // fault-handling tests: block 0 skips its barrier arrivals
  long long spin_limit;  // polls of one barrier wait before it gives up
  // reflected restarted Halpern PDHG (halpern = 1; pdlp_params.halpern): a step maps the
  // Halpern iterate z through the PDHG operator T and mixes z' = ha T(z) + hb z + hc z_a
  // (z_a the anchor); the coefficients of the next step in both precisions, the steps
  // since the last restart (h_k), the reflection rho, the fixed-point residuals of the
  // latest step and of the epoch's first step (prev_cand holds the last check's)
  int halpern, restart_metric;  // restart_metric: 0 KKT_omega, 1 normalized duality gap
  double ndg_last;              // normalized duality gap of the last restart point (A9b)
  long long h_k;
  double h_rho, h_res, h_r0;
  double ha_d, hb_d, hc_d;
  float ha_f, hb_f, hc_f, hf_pad;
};

// Normalized-duality-gap restarts (restart_metric = 1): the trust-region maximum of the
// gap at each candidate, by bisection on the step t of z^(t) = proj(z + t M^-1 g):
// one launch of k_ndg_eval per stage -- 0 the radius r and the dual norm N, 1 the test
// of t0 2^63 (t0 = r / N), 2..7 the bisection over the exponent k of t0 2^k, 8..51 the
// halvings of [t0 2^(k-1), t0 2^k], 52 the gap at the final lower end.
constexpr int kNdgKSteps = 6;
constexpr int kNdgHalvings = 44;
constexpr int kNdgStages = 3 + kNdgKSteps + kNdgHalvings;
// LPs with at most this many columns and rows run every stage in one block (one launch)
constexpr int kNdgOneBlock = 4096;
struct NdgCand {
  double r, nrm, t0, a, b, trial, rho;
  int lo, hi, mid, fixed;  // fixed: t stays t0 2^63 (the region's far end is inside the ball)
  int done, pad;           // done: rho is final (r = 0 or N = 0: rho = 0)
};
struct NdgState {
  NdgCand c[2];  // current, average
  int stage;
  unsigned ticket;  // blocks of the running launch that have added their partials
};

// Halpern variant: passes of the power iteration for ||K~||_2 and the step size's
// fraction of 1 / ||K~||_2
constexpr int kPowerIters = 64;
constexpr double kHalpernEtaScale = 0.998;

// Halpern coefficients of step k = h_k since the last restart:
// lambda = (k + 1) / (k + 2), ha = lambda (1 + rho), hb = -lambda rho, hc = 1 - lambda
__host__ __device__ inline void halpern_coeffs(DevState* st) {
  const double k = (double)st->h_k;
  const double lam = (k + 1.0) / (k + 2.0);
  st->ha_d = lam * (1.0 + st->h_rho);
  st->hb_d = -lam * st->h_rho;
  st->hc_d = 1.0 - lam;
  st->ha_f = (float)st->ha_d;
  st->hb_f = (float)st->hb_d;
  st->hc_f = (float)st->hc_d;
}

// status value of a persistent step kernel whose bounded barrier wait gave up
constexpr int kStatusWaitFailed = 99;
// polls of one grid-barrier wait (seconds at L2 latency); fault-handling tests use 2^16
constexpr long long kSpinLimit = 1LL << 23;
constexpr long long kSpinLimitTest = 1LL << 16;

// ---------------------------------------------------------------- batches
// Launch tables of a batch of LPs solved together (all NULL for one LP): the
// batch is one block-diagonal problem with global row/column indices; every
// block of a kernel belongs to one LP and processes that LP's rows only.
struct Tables {
  const int* blk_lp;  // [grid] block -> LP
  const int* blk0;    // [count] first block of the LP (also its first partial slot)
  const int* nshort;  // [count] blocks over short rows
  const int* nblk;    // [count] all blocks of the LP (short + one per long row)
  const int* row0;    // [count] first global row of the LP in this matrix
  const int* nrows;   // [count] rows of the LP in this matrix
  const int* long0;   // [count] first entry of the LP in the long-row list
  const int* nlong;   // [count] long rows of the LP
};

// The rows of one LP and the blocks that own them, as seen by one block.
struct Span {
  int lp;            // LP index (0 for a single LP)
  int row0, nrows;   // global row range
  int bidx;          // block index within the LP's blocks
  int nshort, nblk;  // the LP's short-row blocks and all its blocks
  int part0;         // global index of the LP's first block (its first partial slot)
  const int* list;   // the LP's long rows (global ids)
  int nlist;
};

// The span of virtual block `vb` of a batch's launch map (the persistent batch kernel
// walks the map's blocks with a resident grid).
__device__ __forceinline__ Span span_of(const Tables& t, int vb, const int* list1) {
  Span s;
  const int k = t.blk_lp[vb];
  s.lp = k;
  s.row0 = t.row0[k];
  s.nrows = t.nrows[k];
  s.part0 = t.blk0[k];
  s.bidx = vb - s.part0;
  s.nshort = t.nshort[k];
  s.nblk = t.nblk[k];
  s.list = list1 + t.long0[k];
  s.nlist = t.nlong[k];
  return s;
}

__device__ __forceinline__ Span make_span(const Tables& t, int nrows1, int nshort1,
                                          const int* list1, int nlist1) {
  Span s;
  if (t.blk_lp == nullptr) {
    s.lp = 0;
    s.row0 = 0;
    s.nrows = nrows1;
    // the long-row blocks (the grid's last gridDim.x - nshort1 logical blocks) take the
    // lowest block indices, so that they are scheduled first and their long loops
    // overlap the short rows instead of trailing behind them
    const int nl = (int)gridDim.x - nshort1;
    s.bidx = (int)blockIdx.x < nl ? nshort1 + (int)blockIdx.x : (int)blockIdx.x - nl;
    s.nshort = nshort1;
    s.nblk = gridDim.x;
    s.part0 = 0;
    s.list = list1;
    s.nlist = nlist1;
  } else {
    const int k = t.blk_lp[blockIdx.x];
    s.lp = k;
    s.row0 = t.row0[k];
    s.nrows = t.nrows[k];
    s.part0 = t.blk0[k];
    s.bidx = blockIdx.x - s.part0;
    s.nshort = t.nshort[k];
    s.nblk = t.nblk[k];
    s.list = list1 + t.long0[k];
    s.nlist = t.nlong[k];
  }
  return s;
}

// ---------------------------------------------------------------- tiles
// Work items of the staged tile step kernels (tile_kernels.cuh), built at setup
// (setup_tiles).  A tile is a run of at most kTileRows consecutive rows of at
// most kLongRow entries whose nonzeros start inside one window of W entries
// (kTileWindowMin <= W <= kTileWindowMax); a longer row is cut into slices of at
// most W entries.  No item straddles two LPs of a batch.
constexpr int kTileRows = kBlock;
constexpr int kLongRow = 256;
constexpr int kTileWindowMin = 256;
constexpr int kTileWindowMax = 1024;
// warp tiles (wtile_kernels.cuh): at most 32 rows, windows of 64-256 nonzeros
constexpr int kWarpTileRows = 32;
constexpr int kWarpTileWindowMin = 64;
constexpr int kWarpTileWindowMax = 256;

// One work item (32 bytes).  Tile: rows [r0, r1), nonzeros [nb, ne), first = -1.
// Slice: row r0 (r1 = r0 + 1), nonzeros [nb, ne) of it, first = index of the row's
// first slice, nsl = slices of the row, lid = the row's long-row slot.
struct TileItem {
  int r0, r1, nb, ne;
  int lp, first, nsl, lid;
};

// Item tables of one orientation and the slots the kernels write.
struct TileSet {
  const TileItem* item;  // [n]
  int n;                 // items
  const int* item0;      // [count + 1] first item of each LP
  const int* lng0;       // [count + 1] first long-row slot of each LP
  float2* part;          // [n x kWarps] per-(block, LP) partial sums of each warp, in the slot
                         // of the run's first item
  float2* rowpart;       // [n] a slice's partial row sum(s)
  float2* lterm;         // [long rows] a finished long row's partial-sum terms
  int* ticket;           // [n] slices done, in the slot of a row's first slice (0 between launches)
};

// ---------------------------------------------------------------- dependent launch
// Programmatic dependent launch: kernels of the iteration chain are launched
// with the programmatic-serialization attribute, so the next kernel's blocks
// are scheduled while this one drains.  Every such kernel waits for its
// predecessor grid (completion and memory flush) before it reads anything,
// then lets its own dependents launch.  Launched without the attribute, both
// instructions return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_launch_dependents();
}

// ---------------------------------------------------------------- reductions
template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T v) {
  // sum over an aligned group of LANES lanes; all lanes of the group are active
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = (LANES == 32) ? 0xffffffffu : (((1u << LANES) - 1u) << (lane & ~(unsigned)(LANES - 1)));
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// pair of partial sums reduced together (two candidates, or x' and dx)
template <typename T>
struct P2 {
  T a, b;
  __device__ __forceinline__ P2& operator+=(const P2& o) {
    a += o.a;
    b += o.b;
    return *this;
  }
};
using D2 = P2<double>;
template <int LANES, typename T>
__device__ __forceinline__ P2<T> group_sum(P2<T> v) {
  v.a = group_sum<LANES, T>(v.a);
  v.b = group_sum<LANES, T>(v.b);
  return v;
}

// three partial sums reduced together (two candidates and a ray)
struct D3 {
  double a, b, c;
  __device__ __forceinline__ D3& operator+=(const D3& o) {
    a += o.a;
    b += o.b;
    c += o.c;
    return *this;
  }
};
template <int LANES>
__device__ __forceinline__ D3 group_sum(D3 v) {
  v.a = group_sum<LANES, double>(v.a);
  v.b = group_sum<LANES, double>(v.b);
  v.c = group_sum<LANES, double>(v.c);
  return v;
}

// interleaved (value, step) pairs of the primal iterate: .x = x_j, .y = x_j - x_j(previous)
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using vec2_t = typename Vec2<T>::type;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic sum of NV values over a block of kBlock threads.  Thread 0
// gets the result; the order of additions is fixed by the launch shape.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (&out)[NV]) {
  __shared__ double sh[NV][kWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = warp_sum(v[k]);
    if (lane == 0) sh[k][w] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int i = 0; i < kWarps; ++i) s += sh[k][i];
      out[k] = s;
    }
  }
  __syncthreads();
}

// Deterministic sum of NV <= 16 float64 values over a block, thread 0 gets the
// result.  Within a warp a reduce-scatter: at each of the offsets 16, 8, 4, 2 a
// lane keeps the half of its values its offset bit selects and adds the partner's
// copy of that half, so 8 + 4 + 2 + 1 (+ 1 at offset 1) float64 additions per lane
// replace 5 NV shuffle-additions (a float64 warp instruction holds GB300's float64
// pipe ~16 cycles however many lanes it uses); then one thread per value adds the
// warps' totals in warp order.
template <int NV>
__device__ __forceinline__ void block_sum_rs(const double (&v)[NV], double (&out)[NV]) {
  static_assert(NV >= 1 && NV <= 16, "block_sum_rs takes at most 16 values");
  __shared__ double sh[kWarps][16];
  __shared__ double res[16];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double a[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = k < NV ? v[k] : 0.0;
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double send = hi ? a[k] : a[k + h];
      const double keep = hi ? a[k + h] : a[k];
      a[k] = keep + __shfl_xor_sync(full, send, o);
    }
  }
  a[0] += __shfl_xor_sync(full, a[0], 1);
  // lanes L and L ^ 1 now hold the warp total of value 8 b4 + 4 b3 + 2 b2 + b1 (b_i = bit i of L)
  if ((lane & 1) == 0) sh[w][((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                          ((lane >> 1) & 1)] = a[0];
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int i = 0; i < kWarps; ++i) t += sh[i][threadIdx.x];
    res[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = res[k];
  }
  __syncthreads();
}

// Deterministic block sum in the element type T (float reductions stay in the
// float32 pipe); thread 0 gets the result.
template <typename T>
__device__ __forceinline__ T block_sum1(T v) {
  __shared__ T sh[kWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kWarps; ++i) s += sh[i];
  __syncthreads();
  return s;
}

// Three sums at once (one shared-memory round instead of three); thread 0 gets them.
template <typename T>
__device__ __forceinline__ void block_sum3(T& a, T& b, T& c) {
  __shared__ T sh[3][kWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][w] = a;
    sh[1][w] = b;
    sh[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0;
    for (int i = 0; i < kWarps; ++i) {
      a += sh[0][i];
      b += sh[1][i];
      c += sh[2][i];
    }
  }
}

// Fixed-order reduction of NV partial arrays part[k * stride + i], i < count,
// by one block; thread 0 receives the sums.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* part, int stride, int count,
                                                double (&out)[NV]) {
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int i = threadIdx.x; i < count; i += kBlock) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += part[(size_t)k * stride + i];
  }
  block_sum_rs<NV>(v, out);
}

__device__ __forceinline__ double kkt_omega(double omega, double rp2, double rd2, double gap2) {
  return sqrt(omega * rp2 + rd2 / omega + gap2);
}

}  // namespace pdlp
