// Device setup of one LP (rows A0-A3 of the hot path):
//   validation of the caller's CSR and vectors (error bits, no trap),
//   canonical form K = S A, q = S b (A0),
//   deterministic transpose of A into CSR (A1: count, scan, scatter, then a
//   segmented sort of each column's entries by their position in A, so the
//   result does not depend on the order atomics landed in),
//   Ruiz (inf-norm) and Pock-Chambolle scaling (A2),
//   iteration-space matrix values and vectors, and the scalars of A3.
#include <algorithm>
#include <vector>

#include "setup.h"

namespace pdlp {

namespace {

constexpr int kScanItems = 8;                       // per thread
constexpr int kScanTile = kBlock * kScanItems;      // per block
constexpr int kSmallSeg = 32;                       // per-thread insertion sort up to this length
constexpr int kTile = 4096;                         // bitonic tile of a long column segment

// ------------------------------------------------------------------ validation
__global__ void k_validate_rows(SetupIn in, int* err) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < in.m; i += stride) {
    const int64_t s = in.row_ptr[i], e = in.row_ptr[i + 1];
    if (s < 0 || e < s || e > in.nnz) atomicOr(err, ERR_ROWPTR);
    const char sn = in.sense[i];
    if (sn != 'L' && sn != 'G' && sn != 'E') atomicOr(err, ERR_SENSE);
    if (!isfinite(in.b[i])) atomicOr(err, ERR_NONFINITE);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (in.row_ptr[0] != 0 || in.row_ptr[in.m] != in.nnz) atomicOr(err, ERR_ROWPTR);
  }
}

__global__ void k_validate_nnz(SetupIn in, int* err) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < in.nnz; p += stride) {
    const int j = in.col[p];
    if (j < 0 || j >= in.n) atomicOr(err, ERR_COL);
    if (!isfinite(in.val[p])) atomicOr(err, ERR_NONFINITE);
  }
}

__global__ void k_validate_cols(SetupIn in, int* err) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < in.n; j += stride) {
    const double l = in.l[j], u = in.u[j];
    if (!isfinite(in.c[j])) atomicOr(err, ERR_NONFINITE);
    if (isnan(l) || isnan(u) || l > u || l == INFINITY || u == -INFINITY) atomicOr(err, ERR_BOUNDS);
  }
}

// ------------------------------------------------------------------ A0
__global__ void k_canonical(SetupIn in, int* a_ptr, int* a_col, double* a_val64, double* q,
                            unsigned char* row_kind) {
  // one warp per row
  const int lane = threadIdx.x & 31;
  const long long W = (long long)gridDim.x * blockDim.x / 32;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < in.m; i += W) {
    const char sn = in.sense[i];
    const double s = sn == 'L' ? -1.0 : 1.0;
    const int64_t b = in.row_ptr[i], e = in.row_ptr[i + 1];
    for (int64_t p = b + lane; p < e; p += 32) {
      a_col[p] = in.col[p];
      a_val64[p] = s * in.val[p];
    }
    if (lane == 0) {
      a_ptr[i] = (int)b;
      q[i] = s * in.b[i];
      row_kind[i] = sn == 'E' ? 1 : (sn == 'L' ? 2 : 0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a_ptr[in.m] = (int)in.nnz;
}

// ------------------------------------------------------------------ scan
// exclusive scan of cnt[0..N) into out[0..N], out[N] = total
__global__ void k_scan_tiles(const int* cnt, int* out, int N, int* bsum) {
  __shared__ int sh[kBlock];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    v[k] = i < N ? cnt[i] : 0;
    s += v[k];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < kBlock; o <<= 1) {  // Hillis-Steele inclusive scan of thread sums
    const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - s;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    if (i < N) out[i] = run;
    run += v[k];
  }
  if (threadIdx.x == kBlock - 1) bsum[blockIdx.x] = sh[kBlock - 1];
}

__global__ void k_scan_bsum(int* bsum, int nb, int* out, int N) {
  // single block: exclusive scan of the tile sums, written back in place; total into out[N]
  __shared__ int sh[kBlock];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += kBlock) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kBlock; o <<= 1) {
      const int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) bsum[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kBlock - 1) carry += sh[kBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[N] = carry;
}

__global__ void k_scan_add(int* out, int N, const int* bsum) {
  const long long base = (long long)blockIdx.x * kScanTile;
  const int add = bsum[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += kBlock) {
    const long long i = base + k;
    if (i < N) out[i] += add;
  }
}

// ------------------------------------------------------------------ A1 transpose
__global__ void k_count_cols(const int* a_col, int nnz, int* cnt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
    atomicAdd(cnt + a_col[p], 1);
}

__global__ void k_scatter(const int* a_col, int nnz, const int* t_ptr, int* cursor, int* src) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int j = a_col[p];
    const int pos = t_ptr[j] + atomicAdd(cursor + j, 1);
    src[pos] = (int)p;
  }
}

__global__ void k_segsort_small(const int* t_ptr, int n, int* src, int* long_list, int* nlong) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    const int s = t_ptr[j], e = t_ptr[j + 1], len = e - s;
    if (len > kSmallSeg) {
      long_list[atomicAdd(nlong, 1)] = (int)j;
      continue;
    }
    int k[kSmallSeg];
    for (int a = 0; a < len; ++a) k[a] = src[s + a];
    for (int a = 1; a < len; ++a) {  // insertion sort
      const int v = k[a];
      int b = a - 1;
      while (b >= 0 && k[b] > v) {
        k[b + 1] = k[b];
        --b;
      }
      k[b + 1] = v;
    }
    for (int a = 0; a < len; ++a) src[s + a] = k[a];
  }
}

// one block per tile (start, len <= kTile): bitonic sort in shared memory, in place
__global__ void __launch_bounds__(1024) k_sort_tiles(const int2* tiles, int* src) {
  __shared__ int sh[kTile];
  const int2 t = tiles[blockIdx.x];
  const int start = t.x, len = t.y;
  int P = 1;
  while (P < len) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? src[start + i] : INT_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ jj;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const int a = sh[i], b = sh[ixj];
          if ((a > b) == up) {
            sh[i] = b;
            sh[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) src[start + i] = sh[i];
}

// segments of more than one sorted tile: the rank of a key is its index in its
// tile plus the number of smaller keys in every other tile of the segment
// (keys are unique positions in A)
__global__ void k_merge_rank(const int4* mtiles, const int* src, int* out) {
  // mtiles[b] = {seg_start, seg_len, tile_start, tile_len}
  const int4 t = mtiles[blockIdx.x];
  const int seg_s = t.x, seg_len = t.y, ts = t.z, tl = t.w;
  for (int i = threadIdx.x; i < tl; i += blockDim.x) {
    const int key = src[ts + i];
    int rank = i;
    for (int o = seg_s; o < seg_s + seg_len; o += kTile) {
      if (o == ts) continue;
      const int ol = min(kTile, seg_s + seg_len - o);
      int lo = 0, hi = ol;  // count of keys < key in sorted [o, o+ol)
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (src[o + mid] < key) lo = mid + 1;
        else hi = mid;
      }
      rank += lo;
    }
    out[seg_s + rank] = key;
  }
}

__global__ void k_copy_ranges(const int2* ranges, const int* from, int* to) {
  const int2 r = ranges[blockIdx.x];
  for (int i = threadIdx.x; i < r.y; i += blockDim.x) to[r.x + i] = from[r.x + i];
}

// Tile descriptors of the long column segments built on the device (used when
// the caller cannot let the host allocate): per segment its tile count and, for
// segments longer than one tile, the merge-rank tile count.
__global__ void k_tile_counts(const int* list, int nlist, const int* t_ptr, int* cnt_t, int* cnt_m) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nlist; k += stride) {
    const int j = list[k];
    const int len = t_ptr[j + 1] - t_ptr[j];
    const int tiles = (len + kTile - 1) / kTile;
    cnt_t[k] = tiles;
    cnt_m[k] = len > kTile ? tiles : 0;
  }
}

__global__ void k_tile_desc(const int* list, int nlist, const int* t_ptr, const int* off_t,
                            const int* off_m, int2* tiles, int4* mtiles, int2* ranges) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nlist; k += stride) {
    const int j = list[k];
    const int st = t_ptr[j], len = t_ptr[j + 1] - st;
    int a = off_t[k], b = off_m[k];
    for (int o = 0; o < len; o += kTile) {
      const int tl = min(kTile, len - o);
      tiles[a++] = make_int2(st + o, tl);
      if (len > kTile) mtiles[b++] = make_int4(st, len, st + o, tl);
    }
    ranges[k] = make_int2(st, len > kTile ? len : 0);
  }
}

__global__ void k_finish_transpose(const int* a_ptr, int m, const double* a_val64, const int* src,
                                   int nnz, int* t_col, double* t_val64) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int s = src[p];
    int lo = 0, hi = m;  // last row whose start <= s
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a_ptr[mid] <= s) lo = mid;
      else hi = mid - 1;
    }
    t_col[p] = lo;
    t_val64[p] = a_val64[s];
  }
}

// ------------------------------------------------------------------ A2 scaling
// row statistics of |K~_ij| = (dr_i |K_ij|) dc_j over a CSR orientation:
// op 0 = max, op 1 = sum of |K~|^power.  In the A^T orientation the roles of
// the two scale vectors swap (rowscale = dc, colscale = dr) but the product is
// formed in the same order as in A: (dr_i |K_ij|) dc_j.
// Row statistics of the scaled matrix D_own K D_other (one group of LANES lanes
// per row): op 0 the max of |k~_ij|, op 1 the sum of |k~_ij|^power.  Float64
// throughout (the scaling feeds the float64 parity mode); on GB300 a float64
// warp instruction costs the FP64 pipe ~16 cycles whatever the active lanes,
// so a short row gets few lanes instead of a whole warp.
template <int LANES>
__device__ __forceinline__ void rowstat_rows(const int* ptr, const int* col, const double* val,
                                             int nrows, const double* own, const double* other,
                                             int own_is_row, int op, double power, double* out,
                                             int bidx, int nblk) {
  const int lane = threadIdx.x & (LANES - 1);
  const long long G = (long long)nblk * blockDim.x / LANES;
  for (long long r = ((long long)bidx * blockDim.x + threadIdx.x) / LANES; r < nrows; r += G) {
    const int s = ptr[r], e = ptr[r + 1];
    const double so = own[r];
    double acc = 0.0;
    for (int p = s + lane; p < e; p += LANES) {
      const double a = fabs(val[p]);
      const double o = other[col[p]];
      // (D_r |K|) D_c rounded product by product, never fused into an add
      const double kt = own_is_row ? __dmul_rn(__dmul_rn(so, a), o) : __dmul_rn(__dmul_rn(o, a), so);
      if (op == 0) acc = fmax(acc, kt);
      else acc = __dadd_rn(acc, power == 1.0 ? kt : pow(kt, power));
    }
    const unsigned mask = LANES == 32 ? 0xffffffffu
                                      : (((1u << LANES) - 1u) << ((threadIdx.x & 31) & ~(LANES - 1)));
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) {
      const double t = __shfl_xor_sync(mask, acc, o);
      acc = op == 0 ? fmax(acc, t) : acc + t;
    }
    if (lane == 0) out[r] = acc;
  }
}

// One statistics pass of the scaling over both orientations in one launch: blocks
// [0, ga) take the rows of A (row statistics), the rest the rows of A^T (column
// statistics); the two halves read the same D_r, D_c and run side by side.
struct StatPass {
  const int *a_ptr, *a_col, *t_ptr, *t_col;
  const double *a_val, *t_val, *dr, *dc;
  int m, n, ga, op;
  double pow_r, pow_c;
  double *stat_r, *stat_c;
};

template <int LA, int LT>
__global__ void k_stat_pass(StatPass q) {
  pdl_enter();
  if ((int)blockIdx.x < q.ga)
    rowstat_rows<LA>(q.a_ptr, q.a_col, q.a_val, q.m, q.dr, q.dc, 1, q.op, q.pow_r, q.stat_r,
                     blockIdx.x, q.ga);
  else
    rowstat_rows<LT>(q.t_ptr, q.t_col, q.t_val, q.n, q.dc, q.dr, 0, q.op, q.pow_c, q.stat_c,
                     blockIdx.x - q.ga, gridDim.x - q.ga);
}

// D_r /= sqrt(stat_r), D_c /= sqrt(stat_c) (a zero statistic leaves the factor)
__global__ void k_apply_scale2(double* dr, const double* stat_r, int m, double* dc,
                               const double* stat_c, int n) {
  pdl_enter();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)m + n;
       i += stride) {
    double* d = i < m ? dr + i : dc + (i - m);
    const double st = i < m ? stat_r[i] : stat_c[i - m];
    *d = *d / (st > 0.0 ? sqrt(st) : 1.0);
  }
}

// lanes per row for an average row length (about four entries per lane)
static int stat_lanes(double avg) {
  int l = 2;
  while (l < 32 && 4.0 * l < avg) l <<= 1;
  return l;
}

template <int LA>
static cudaError_t stat_pass_la(int lt, int grid, const StatPass& q, cudaStream_t s) {
  switch (lt) {
    case 1: return launch_pdl(k_stat_pass<LA, 1>, grid, kBlock, s, q);
    case 2: return launch_pdl(k_stat_pass<LA, 2>, grid, kBlock, s, q);
    case 4: return launch_pdl(k_stat_pass<LA, 4>, grid, kBlock, s, q);
    case 8: return launch_pdl(k_stat_pass<LA, 8>, grid, kBlock, s, q);
    case 16: return launch_pdl(k_stat_pass<LA, 16>, grid, kBlock, s, q);
    default: return launch_pdl(k_stat_pass<LA, 32>, grid, kBlock, s, q);
  }
}

// one statistics pass (op 0: max |K~|, op 1: sum |K~|^pow) over A and A^T, then
// the application of both scale vectors.  A maximum is exact in any order; a sum
// runs one thread per row over the entries in storage order (rows of A by column,
// rows of A^T by row), the order of a sequential CSR row sum, so that the
// Pock-Chambolle factors round exactly as a plain sequential sum does.
static cudaError_t stat_pass(const ScaleIn& sc, double* dr, double* dc, double* stat_r,
                             double* stat_c, int op, double pow_r, double pow_c, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  const int la = op == 1 ? 1 : stat_lanes(sc.m > 0 ? (double)sc.nnz / sc.m : 1.0);
  const int lt = op == 1 ? 1 : stat_lanes((double)sc.nnz / sc.n);
  const int ga = sc.m > 0 ? grid_for((long long)sc.m * la, G) : 0;
  const int gt = grid_for((long long)sc.n * lt, G);
  const StatPass q{sc.a_ptr, sc.a_col, sc.t_ptr, sc.t_col, sc.a_val64, sc.t_val64, dr, dc,
                   sc.m, sc.n, ga, op, pow_r, pow_c, stat_r, stat_c};
  cudaError_t e;
  switch (la) {
    case 1: e = stat_pass_la<1>(lt, ga + gt, q, s); break;
    case 2: e = stat_pass_la<2>(lt, ga + gt, q, s); break;
    case 4: e = stat_pass_la<4>(lt, ga + gt, q, s); break;
    case 8: e = stat_pass_la<8>(lt, ga + gt, q, s); break;
    case 16: e = stat_pass_la<16>(lt, ga + gt, q, s); break;
    default: e = stat_pass_la<32>(lt, ga + gt, q, s); break;
  }
  if (e != cudaSuccess) return e;
  return launch_pdl(k_apply_scale2, grid_for((long long)sc.m + sc.n, G), kBlock, s, dr, stat_r,
                    sc.m, dc, stat_c, sc.n);
}

__global__ void k_fill(double* p, double v, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

// ------------------------------------------------------------------ value formats
__global__ void k_value_format(const double* val, int nnz, int* flags) {
  // flags[0] &= every value exactly representable in bfloat16; flags[1] &= every value == 1
  bool bf = true, one = true;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const double v = val[p];
    bf &= (double)__bfloat162float(__double2bfloat16(v)) == v;
    one &= v == 1.0;
  }
  if (!__all_sync(0xffffffffu, bf) && (threadIdx.x & 31) == 0) atomicAnd(flags, 0);
  if (!__all_sync(0xffffffffu, one) && (threadIdx.x & 31) == 0) atomicAnd(flags + 1, 0);
}

// iteration matrix values: scaled (dr_i K_ij) dc_j or raw K_ij, in both orientations
template <typename V>
__global__ void k_iter_values(const int* ptr, const int* col, const double* val64, int nrows,
                              const double* own, const double* other, int own_is_row, int scaled,
                              V* out) {
  const int lane = threadIdx.x & 31;
  const long long W = (long long)gridDim.x * blockDim.x / 32;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < nrows; r += W) {
    const int s = ptr[r], e = ptr[r + 1];
    const double so = own[r];
    for (int p = s + lane; p < e; p += 32) {
      double v = val64[p];
      if (scaled) {
        const double o = other[col[p]];
        v = own_is_row ? (so * v) * o : (o * v) * so;
      }
      out[p] = (V)v;
    }
  }
}
template <>
__global__ void k_iter_values<__nv_bfloat16>(const int* ptr, const int* col, const double* val64,
                                            int nrows, const double* own, const double* other,
                                            int own_is_row, int scaled, __nv_bfloat16* out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long nnz = ptr[nrows];
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
    out[p] = __double2bfloat16(val64[p]);
}

// iteration-space vectors (A2/A3) and the float64 scalars of A3
template <typename T>
__global__ void k_iter_vectors(VecIn v, T* c, T* l, T* u, T* q, T* tw, T* sw, T* x0, T* y0,
                               double* part) {
  // part[b*7 + k]: k = 0 ||D_c c||^2, 1 ||D_r q||^2, 2 ||c||^2, 3 ||q||^2, 4 ||x~_hint||^2,
  // 5 ||y~_hint||^2 (the hint projected like a start, in scaled space), 6 columns with
  // an infinite bound
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < v.n; j += stride) {
    const double d = v.dc[j], cj = v.c[j];
    double lj = v.l[j], uj = v.u[j];
    if (v.scaled) {
      c[j] = (T)(d * cj);
      lj = lj / d;
      uj = uj / d;
    } else {
      c[j] = (T)cj;
      tw[j] = (T)(d * d);
    }
    l[j] = (T)lj;
    u[j] = (T)uj;
    double x = v.x0 ? (v.scaled ? v.x0[j] / d : v.x0[j]) : 0.0;
    x = fmin(fmax(x, lj), uj);
    x0[2 * j] = (T)x;  // (x_j, dx_j) pair, no step yet
    x0[2 * j + 1] = (T)0;
    acc[0] += (d * cj) * (d * cj);
    acc[2] += cj * cj;
    acc[6] += (isfinite(v.l[j]) && isfinite(v.u[j])) ? 0.0 : 1.0;
    if (v.wx) {
      const double xh = fmin(fmax(v.wx[j] / d, v.l[j] / d), v.u[j] / d);
      acc[4] += xh * xh;
    }
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < v.m; i += stride) {
    const double d = v.dr[i], qi = v.q[i];
    if (v.scaled) {
      q[i] = (T)(d * qi);
    } else {
      q[i] = (T)qi;
      sw[i] = (T)(d * d);
    }
    double y = 0.0;
    if (v.y0) {
      const double yc = v.row_kind[i] == 2 ? -v.y0[i] : v.y0[i];  // caller convention -> canonical
      y = v.scaled ? yc / d : yc;
      if (v.row_kind[i] != 1) y = fmax(y, 0.0);
    }
    y0[i] = (T)y;
    acc[1] += (d * qi) * (d * qi);
    acc[3] += qi * qi;
    if (v.wy) {
      double yh = (v.row_kind[i] == 2 ? -v.wy[i] : v.wy[i]) / d;
      if (v.row_kind[i] != 1) yh = fmax(yh, 0.0);
      acc[5] += yh * yh;
    }
  }
  double out[7];
  block_sum<7>(acc, out);
  if (threadIdx.x == 0)
    for (int k = 0; k < 7; ++k) part[(size_t)blockIdx.x * 7 + k] = out[k];
}

__global__ void k_absmax_scaled(const int* ptr, const int* col, const double* val64, int nrows,
                                const double* dr, const double* dc, double* part) {
  double mx = 0.0;
  const int lane = threadIdx.x & 31;
  const long long W = (long long)gridDim.x * blockDim.x / 32;
  for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < nrows; r += W) {
    const int s = ptr[r], e = ptr[r + 1];
    for (int p = s + lane; p < e; p += 32) mx = fmax(mx, fabs((dr[r] * val64[p]) * dc[col[p]]));
  }
  __shared__ double sh[kWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kWarps; ++i) mx = fmax(mx, sh[i]);
    part[blockIdx.x] = mx;
  }
}

__global__ void k_finish_scalars(const double* vpart, int nv, const double* mpart, int nmx,
                                 double* out) {
  // out: [0] ||c~||, [1] ||q~||, [2] ||c||, [3] ||q||, [4] max |K~|, [5] ||x~_hint||,
  // [6] ||y~_hint||, [7] columns with an infinite bound
  double a[7] = {0, 0, 0, 0, 0, 0, 0}, r[7];
  for (int b = threadIdx.x; b < nv; b += kBlock)
    for (int k = 0; k < 7; ++k) a[k] += vpart[(size_t)b * 7 + k];
  block_sum<7>(a, r);
  __shared__ double mx;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int b = 0; b < nmx; ++b) m = fmax(m, mpart[b]);
    mx = m;
    for (int k = 0; k < 4; ++k) out[k] = sqrt(r[k]);
    out[4] = mx;
    out[5] = sqrt(r[4]);
    out[6] = sqrt(r[5]);
    out[7] = r[6];
  }
}

// Bound-objective rescaling (optional, after A2/A3's vectors): the iteration-space
// objective divided by gamma, the right-hand side, the bounds and the start x by beta,
// the start y by gamma; the factors that carry an iteration-space point back to the
// original units (D_c, D_r of the KKT passes and the output) take beta and gamma in,
// and their inverses (the scaled distances of the primal-weight update) 1 / beta and
// 1 / gamma.  The step weights and the iteration matrix were formed before and keep
// the plain D_r, D_c.
template <typename T>
__global__ void k_rescale(int m, int n, double beta, double gamma, T* c, T* l, T* u, T* q, T* x0,
                          T* y0, double* dr, double* dc, double* inv_dr, double* inv_dc) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    c[j] = (T)((double)c[j] / gamma);
    l[j] = (T)((double)l[j] / beta);
    u[j] = (T)((double)u[j] / beta);
    x0[2 * j] = (T)((double)x0[2 * j] / beta);
    dc[j] = dc[j] * beta;
    inv_dc[j] = 1.0 / dc[j];
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    q[i] = (T)((double)q[i] / beta);
    y0[i] = (T)((double)y0[i] / gamma);
    dr[i] = dr[i] * gamma;
    inv_dr[i] = 1.0 / dr[i];
  }
}

// rows by descending length, ties by index: a row's place is the number of rows before it
// in that order (every thread compares its row with all the others)
__global__ void k_len_order(const int* ptr, int rows, int* ord) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
    const int len = ptr[r + 1] - ptr[r];
    int pos = 0;
    for (int k = 0; k < rows; ++k) {
      const int lk = ptr[k + 1] - ptr[k];
      pos += (lk > len) || (lk == len && k < r);
    }
    ord[pos] = (int)r;
  }
}

// float64 auxiliaries of the KKT passes: 1 / D_r, 1 / D_c and, per column, bit 0
// = lower bound finite, bit 1 = upper bound finite (integer tests instead of
// float64 compares in the per-column epilogue)
__global__ void k_kkt_aux(int m, int n, const double* dr, const double* dc, const double* l,
                          const double* u, double* inv_dr, double* inv_dc, unsigned char* bflags) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
    inv_dr[i] = 1.0 / dr[i];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
    inv_dc[j] = 1.0 / dc[j];
    bflags[j] = (unsigned char)((isfinite(l[j]) ? 1 : 0) | (isfinite(u[j]) ? 2 : 0));
  }
}

// deterministic list of rows longer than thresh: flags, scan, scatter
__global__ void k_long_flags(const int* ptr, int nrows, int thresh, int* flags) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride)
    flags[r] = (ptr[r + 1] - ptr[r]) > thresh ? 1 : 0;
}
__global__ void k_long_scatter(const int* flags, const int* pos, int nrows, int* list) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += stride)
    if (flags[r]) list[pos[r]] = (int)r;
}

}  // namespace

int grid_for(long long work_items, int max_blocks) {
  long long g = (work_items + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

#define RET(x)                                  \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return e_;           \
  } while (0)

cudaError_t setup_validate(const SetupIn& in, int* d_err, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  RET(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  k_validate_rows<<<grid_for(in.m + 1, G), kBlock, 0, s>>>(in, d_err);
  RET(cudaGetLastError());
  if (in.nnz > 0) {
    k_validate_nnz<<<grid_for(in.nnz, G), kBlock, 0, s>>>(in, d_err);
    RET(cudaGetLastError());
  }
  k_validate_cols<<<grid_for(in.n, G), kBlock, 0, s>>>(in, d_err);
  return cudaGetLastError();
}

cudaError_t setup_canonical(const SetupIn& in, int* a_ptr, int* a_col, double* a_val64, double* q,
                            unsigned char* row_kind, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  k_canonical<<<grid_for((long long)in.m * 32, G), kBlock, 0, s>>>(in, a_ptr, a_col, a_val64, q,
                                                                    row_kind);
  return cudaGetLastError();
}

cudaError_t exclusive_scan(const int* cnt, int* out, int N, int* bsum, cudaStream_t s) {
  const int nb = (N + kScanTile - 1) / kScanTile;
  if (nb > 0) {
    k_scan_tiles<<<nb, kBlock, 0, s>>>(cnt, out, N, bsum);
    RET(cudaGetLastError());
  }
  k_scan_bsum<<<1, kBlock, 0, s>>>(bsum, nb, out, N);
  RET(cudaGetLastError());
  if (nb > 0) {
    k_scan_add<<<nb, kBlock, 0, s>>>(out, N, bsum);
    RET(cudaGetLastError());
  }
  return cudaSuccess;
}

size_t scan_tmp_ints(long long N) { return (size_t)((N + kScanTile - 1) / kScanTile) + 1; }

cudaError_t setup_transpose(int m, int n, int nnz, const int* a_ptr, const int* a_col,
                            const double* a_val64, int* t_ptr, int* t_col, double* t_val64,
                            int* tmp, cudaStream_t s, bool device_desc) {
  // tmp layout (ints): cnt/cursor [n+1] | src [nnz] | src2 [nnz] | long list [n] | nlong [1]
  //                    | tile descriptors [8 * (nnz/32 + 2)], 16-byte aligned | scan block sums
  const int G = device_sm_count() * 8;
  int* cnt = tmp;
  int* src = cnt + (n + 1);
  int* src2 = src + nnz;
  int* long_list = src2 + nnz;
  int* d_nlong = long_list + n;
  size_t doff = (size_t)(d_nlong + 1 - tmp);
  doff = (doff + 3) & ~(size_t)3;
  int* desc = tmp + doff;
  // bound on tiles of segments longer than 32, rounded up to even so that the
  // int4 array placed after 2 * max_desc ints starts on a 16-byte boundary
  const size_t max_desc = ((size_t)nnz / 32 + 3) & ~(size_t)1;
  int* bsum = desc + 8 * max_desc;
  RET(cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
  if (nnz > 0) {
    k_count_cols<<<grid_for(nnz, G), kBlock, 0, s>>>(a_col, nnz, cnt);
    RET(cudaGetLastError());
  }
  RET(exclusive_scan(cnt, t_ptr, n, bsum, s));
  RET(cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s));
  if (nnz > 0) {
    k_scatter<<<grid_for(nnz, G), kBlock, 0, s>>>(a_col, nnz, t_ptr, cnt, src);
    RET(cudaGetLastError());
  }
  RET(cudaMemsetAsync(d_nlong, 0, sizeof(int), s));
  k_segsort_small<<<grid_for(n, G), kBlock, 0, s>>>(t_ptr, n, src, long_list, d_nlong);
  RET(cudaGetLastError());
  int nlong = 0;
  RET(cudaMemcpyAsync(&nlong, d_nlong, sizeof(int), cudaMemcpyDeviceToHost, s));
  RET(cudaStreamSynchronize(s));
  if (nlong > 0 && device_desc) {
    // descriptors built on the device; the count and offset arrays live in src2,
    // which the merge-rank pass only overwrites after the descriptors exist
    int* cnt_t = src2;
    int* cnt_m = cnt_t + nlong;
    int* off_t = cnt_m + nlong;
    int* off_m = off_t + nlong + 1;
    const int gl = grid_for(nlong, G);
    k_tile_counts<<<gl, kBlock, 0, s>>>(long_list, nlong, t_ptr, cnt_t, cnt_m);
    RET(cudaGetLastError());
    RET(exclusive_scan(cnt_t, off_t, nlong, bsum, s));
    RET(exclusive_scan(cnt_m, off_m, nlong, bsum, s));
    int tot_t = 0, tot_m = 0;
    RET(cudaMemcpyAsync(&tot_t, off_t + nlong, sizeof(int), cudaMemcpyDeviceToHost, s));
    RET(cudaMemcpyAsync(&tot_m, off_m + nlong, sizeof(int), cudaMemcpyDeviceToHost, s));
    RET(cudaStreamSynchronize(s));
    if ((size_t)tot_t > max_desc || (size_t)tot_m > max_desc || (size_t)nlong > max_desc)
      return cudaErrorInvalidValue;
    int2* d_tiles = (int2*)desc;
    int4* d_mtiles = (int4*)(desc + 2 * max_desc);
    int2* d_ranges = (int2*)(desc + 6 * max_desc);
    k_tile_desc<<<gl, kBlock, 0, s>>>(long_list, nlong, t_ptr, off_t, off_m, d_tiles, d_mtiles,
                                      d_ranges);
    RET(cudaGetLastError());
    k_sort_tiles<<<tot_t, 1024, 0, s>>>(d_tiles, src);
    RET(cudaGetLastError());
    if (tot_m > 0) {
      k_merge_rank<<<tot_m, kBlock, 0, s>>>(d_mtiles, src, src2);
      RET(cudaGetLastError());
      k_copy_ranges<<<nlong, kBlock, 0, s>>>(d_ranges, src2, src);
      RET(cudaGetLastError());
    }
  } else if (nlong > 0) {
    std::vector<int> ids(nlong);
    RET(cudaMemcpyAsync(ids.data(), long_list, sizeof(int) * nlong, cudaMemcpyDeviceToHost, s));
    std::vector<int> hp(n + 1);
    RET(cudaMemcpyAsync(hp.data(), t_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
    RET(cudaStreamSynchronize(s));
    std::sort(ids.begin(), ids.end());
    std::vector<int2> tiles;
    std::vector<int4> mtiles;
    std::vector<int2> mranges;
    for (int j : ids) {
      const int st = hp[j], len = hp[j + 1] - hp[j];
      for (int o = 0; o < len; o += kTile) tiles.push_back(make_int2(st + o, std::min(kTile, len - o)));
      if (len > kTile) {
        for (int o = 0; o < len; o += kTile)
          mtiles.push_back(make_int4(st, len, st + o, std::min(kTile, len - o)));
        mranges.push_back(make_int2(st, len));
      }
    }
    if (tiles.size() > max_desc || mtiles.size() > max_desc) return cudaErrorInvalidValue;
    int2* d_tiles = (int2*)desc;                       // 2 ints each
    int4* d_mtiles = (int4*)(desc + 2 * max_desc);     // 4 ints each
    int2* d_ranges = (int2*)(desc + 6 * max_desc);     // 2 ints each
    RET(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, s));
    if (!mtiles.empty()) {
      RET(cudaMemcpyAsync(d_mtiles, mtiles.data(), sizeof(int4) * mtiles.size(),
                          cudaMemcpyHostToDevice, s));
      RET(cudaMemcpyAsync(d_ranges, mranges.data(), sizeof(int2) * mranges.size(),
                          cudaMemcpyHostToDevice, s));
    }
    k_sort_tiles<<<(int)tiles.size(), 1024, 0, s>>>(d_tiles, src);
    RET(cudaGetLastError());
    if (!mtiles.empty()) {
      k_merge_rank<<<(int)mtiles.size(), kBlock, 0, s>>>(d_mtiles, src, src2);
      RET(cudaGetLastError());
      k_copy_ranges<<<(int)mranges.size(), kBlock, 0, s>>>(d_ranges, src2, src);
      RET(cudaGetLastError());
    }
    // the host vectors are read by the copies above: wait before they go out of scope
    RET(cudaStreamSynchronize(s));
  }
  if (nnz > 0) {
    k_finish_transpose<<<grid_for(nnz, G), kBlock, 0, s>>>(a_ptr, m, a_val64, src, nnz, t_col,
                                                         t_val64);
    RET(cudaGetLastError());
  }
  return cudaSuccess;
}

size_t transpose_tmp_ints(int m, int n, long long nnz) {
  return (size_t)(n + 1) + 2 * (size_t)nnz + (size_t)n + 1 + 4 + 8 * ((size_t)nnz / 32 + 3) +
         scan_tmp_ints((long long)std::max(m, n) + 1) + 64;
}

cudaError_t setup_scaling(const ScaleIn& sc, double* dr, double* dc, double* stat_r,
                          double* stat_c, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  k_fill<<<grid_for(sc.m, G), kBlock, 0, s>>>(dr, 1.0, sc.m);
  RET(cudaGetLastError());
  k_fill<<<grid_for(sc.n, G), kBlock, 0, s>>>(dc, 1.0, sc.n);
  RET(cudaGetLastError());
  for (int it = 0; it < sc.ruiz_iters; ++it)
    RET(stat_pass(sc, dr, dc, stat_r, stat_c, 0, 1.0, 1.0, s));
  if (sc.pc_alpha >= 0.0)
    RET(stat_pass(sc, dr, dc, stat_r, stat_c, 1, 2.0 - sc.pc_alpha, sc.pc_alpha, s));
  return cudaSuccess;
}

cudaError_t setup_value_format(const double* val64, int nnz, int* d_flags, int* h_bf16_exact,
                               int* h_all_one, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  const int ones[2] = {1, 1};
  RET(cudaMemcpyAsync(d_flags, ones, sizeof(ones), cudaMemcpyHostToDevice, s));
  if (nnz > 0) {
    k_value_format<<<grid_for(nnz, G), kBlock, 0, s>>>(val64, nnz, d_flags);
    RET(cudaGetLastError());
  }
  int h[2];
  RET(cudaMemcpyAsync(h, d_flags, sizeof(h), cudaMemcpyDeviceToHost, s));
  RET(cudaStreamSynchronize(s));
  *h_bf16_exact = h[0];
  *h_all_one = h[1];
  return cudaSuccess;
}

cudaError_t setup_iter_values(int which_type, const int* ptr, const int* col, const double* val64,
                              int nrows, const double* own, const double* other, int own_is_row,
                              int scaled, void* out, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  const int g = grid_for((long long)nrows * 32, G);
  switch (which_type) {
    case 0: k_iter_values<double><<<g, kBlock, 0, s>>>(ptr, col, val64, nrows, own, other, own_is_row, scaled, (double*)out); break;
    case 1: k_iter_values<float><<<g, kBlock, 0, s>>>(ptr, col, val64, nrows, own, other, own_is_row, scaled, (float*)out); break;
    case 2: k_iter_values<__nv_bfloat16><<<g, kBlock, 0, s>>>(ptr, col, val64, nrows, own, other, own_is_row, scaled, (__nv_bfloat16*)out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t setup_iter_vectors(const VecIn& v, int fp32, void* c, void* l, void* u, void* q,
                               void* tw, void* sw, void* x0, void* y0, const int* a_ptr,
                               const int* a_col, const double* a_val64, double* part,
                               double* scalars_out, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  const int gv = grid_for(std::max(v.m, v.n), G);
  if (fp32)
    k_iter_vectors<float><<<gv, kBlock, 0, s>>>(v, (float*)c, (float*)l, (float*)u, (float*)q,
                                                (float*)tw, (float*)sw, (float*)x0, (float*)y0, part);
  else
    k_iter_vectors<double><<<gv, kBlock, 0, s>>>(v, (double*)c, (double*)l, (double*)u, (double*)q,
                                                 (double*)tw, (double*)sw, (double*)x0, (double*)y0,
                                                 part);
  RET(cudaGetLastError());
  const int gm = grid_for((long long)v.m * 32, G);
  double* mpart = part + (size_t)gv * 7;
  k_absmax_scaled<<<gm, kBlock, 0, s>>>(a_ptr, a_col, a_val64, v.m, v.dr, v.dc, mpart);
  RET(cudaGetLastError());
  k_finish_scalars<<<1, kBlock, 0, s>>>(part, gv, mpart, gm, scalars_out);
  return cudaGetLastError();
}

size_t setup_part_doubles(int m, int n) {
  const int G = device_sm_count() * 8;
  return (size_t)G * 7 + (size_t)G + 16;
}

// ---- Halpern variant: the power iteration for L ~ ||K~||_2, K~ = D_r K D_c
// (K the canonical matrix; val NULL: every entry +1).  v = w / s is the unit vector of
// the previous pass (w = 1/sqrt(n), s = 1 at the start); a pass forms u = K~ v and
// w = K~^T u, s = ||w||; after the last pass L = sqrt(s).  A zero s leaves v = 0.
__global__ void k_pow_start(double* w, int n, double* s) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const double v = 1.0 / sqrt((double)n);
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) w[j] = v;
  if (blockIdx.x == 0 && threadIdx.x == 0) *s = 1.0;
}

// A pass over the matrix (ptr, col, val): out_r = fo_r sum_p K_rp fi_c(p) in_c(p) / s
// (s NULL: no division), fo, fi the row and column scalings.  Rows of at most `thresh`
// entries by groups of kPowLanes lanes, rows grid-strided (longer rows: k_pow_long); with
// part != NULL also each block's sum of out_r^2 into part[block].
constexpr int kPowLanes = 4;
__device__ __forceinline__ double pow_inv(const double* s) {
  const double sv = s ? *s : 1.0;
  return sv > 0.0 ? 1.0 / sv : 0.0;
}
__device__ __forceinline__ void pow_block_part(double sq, double* part) {
  __shared__ double red[kBlock];
  red[threadIdx.x] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kBlock; k += kPowLanes) t += red[k];  // the groups' first lanes
    part[blockIdx.x] = t;
  }
}
__global__ void __launch_bounds__(kBlock) k_pow_pass(const int* ptr, const int* col,
                                                      const double* val, int rows, int thresh,
                                                      const double* fo, const double* fi,
                                                      const double* in, const double* s,
                                                      double* out, double* part) {
  const int gl = threadIdx.x & (kPowLanes - 1);
  const double inv = pow_inv(s);
  double sq = 0.0;
  const long long G = (long long)gridDim.x * (kBlock / kPowLanes);
  for (long long r = ((long long)blockIdx.x * kBlock + threadIdx.x) / kPowLanes; r < rows; r += G) {
    const int b0 = ptr[r], e0 = ptr[r + 1];
    if (e0 - b0 > thresh) continue;  // uniform within the group
    double acc = 0.0;
    for (int p = b0 + gl; p < e0; p += kPowLanes) {
      const int c = col[p];
      acc += (val ? val[p] : 1.0) * fi[c] * (in[c] * inv);
    }
    acc = group_sum<kPowLanes>(acc);
    if (gl == 0) {
      const double v = fo[r] * acc;
      out[r] = v;
      sq += v * v;
    }
  }
  if (part) pow_block_part(gl == 0 ? sq : 0.0, part);
}
// the rows longer than `thresh` (list[nlist]), one block per row, grid-strided over the list
__global__ void __launch_bounds__(kBlock) k_pow_long(const int* ptr, const int* col,
                                                      const double* val, const int* list,
                                                      int nlist, const double* fo,
                                                      const double* fi, const double* in,
                                                      const double* s, double* out,
                                                      double* part) {
  __shared__ double red[kBlock];
  const double inv = pow_inv(s);
  double sq = 0.0;
  for (int k = blockIdx.x; k < nlist; k += gridDim.x) {
    const int r = list[k];
    double acc = 0.0;
    for (int p = ptr[r] + threadIdx.x; p < ptr[r + 1]; p += kBlock) {
      const int c = col[p];
      acc += (val ? val[p] : 1.0) * fi[c] * (in[c] * inv);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kBlock / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double v = fo[r] * red[0];
      out[r] = v;
      sq += v * v;
    }
    __syncthreads();
  }
  if (part && threadIdx.x == 0) part[blockIdx.x] = sq;
}

// s = sqrt(sum of nb partials), added in slot order (one block)
__global__ void __launch_bounds__(kBlock) k_pow_norm(const double* part, int nb, double* s) {
  __shared__ double red[kBlock];
  double t = 0.0;
  for (int k = threadIdx.x; k < nb; k += kBlock) t += part[k];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *s = sqrt(red[0]);
}

cudaError_t setup_power_norm(const PowIn& q, int iters, double* u, double* w, double* part,
                             int part_cap, double* s_dev, double* L, long long* launches,
                             cudaStream_t s) {
  *L = 0.0;
  const int G = std::max(1, std::min(part_cap / 2, device_sm_count() * 8));
  const int per = kBlock / kPowLanes;
  const int gr = std::max(1, std::min(G, (q.m + per - 1) / per));
  const int gc = std::max(1, std::min(G, (q.n + per - 1) / per));
  const int lr = std::min(q.a_nlong, G), lc = std::min(q.t_nlong, G);
  k_pow_start<<<grid_for(q.n, G), kBlock, 0, s>>>(w, q.n, s_dev);
  *launches += 1;
  for (int it = 0; it < iters; ++it) {
    // u = K~ v over the rows of A, then w = K~^T u over the rows of A^T with ||w||^2
    k_pow_pass<<<gr, kBlock, 0, s>>>(q.a_ptr, q.a_col, q.a_val, q.m, q.a_thresh, q.dr, q.dc, w,
                                     s_dev, u, nullptr);
    if (lr) k_pow_long<<<lr, kBlock, 0, s>>>(q.a_ptr, q.a_col, q.a_val, q.a_long, q.a_nlong, q.dr,
                                             q.dc, w, s_dev, u, nullptr);
    k_pow_pass<<<gc, kBlock, 0, s>>>(q.t_ptr, q.t_col, q.t_val, q.n, q.t_thresh, q.dc, q.dr, u,
                                     nullptr, w, part);
    if (lc) k_pow_long<<<lc, kBlock, 0, s>>>(q.t_ptr, q.t_col, q.t_val, q.t_long, q.t_nlong, q.dc,
                                             q.dr, u, nullptr, w, part + gc);
    k_pow_norm<<<1, kBlock, 0, s>>>(part, gc + lc, s_dev);
    *launches += 3 + (lr ? 1 : 0) + (lc ? 1 : 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double sv = 0.0;
  e = cudaMemcpyAsync(&sv, s_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *L = sqrt(sv);
  return e;
}

cudaError_t setup_len_order(const int* ptr, int rows, int* ord, cudaStream_t s) {
  k_len_order<<<grid_for(rows, device_sm_count() * 8), kBlock, 0, s>>>(ptr, rows, ord);
  return cudaGetLastError();
}

cudaError_t setup_rescale(int m, int n, int fp32, double beta, double gamma, void* c, void* l,
                          void* u, void* q, void* x0, void* y0, double* dr, double* dc,
                          double* inv_dr, double* inv_dc, cudaStream_t s) {
  const int g = grid_for(std::max(m, n), device_sm_count() * 8);
  if (fp32)
    k_rescale<float><<<g, kBlock, 0, s>>>(m, n, beta, gamma, (float*)c, (float*)l, (float*)u,
                                          (float*)q, (float*)x0, (float*)y0, dr, dc, inv_dr, inv_dc);
  else
    k_rescale<double><<<g, kBlock, 0, s>>>(m, n, beta, gamma, (double*)c, (double*)l, (double*)u,
                                           (double*)q, (double*)x0, (double*)y0, dr, dc, inv_dr,
                                           inv_dc);
  return cudaGetLastError();
}

cudaError_t setup_kkt_aux(int m, int n, const double* dr, const double* dc, const double* l,
                          const double* u, double* inv_dr, double* inv_dc, unsigned char* bflags,
                          cudaStream_t s) {
  k_kkt_aux<<<grid_for(std::max(m, n), device_sm_count() * 8), kBlock, 0, s>>>(
      m, n, dr, dc, l, u, inv_dr, inv_dc, bflags);
  return cudaGetLastError();
}

__global__ void k_offset_copy(int* dst, const int* src, long long count, int offset) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    dst[i] = src[i] + offset;
}

cudaError_t setup_offset_copy(int* dst, const int* src, long long count, int offset,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_offset_copy<<<grid_for(count, device_sm_count() * 8), kBlock, 0, s>>>(dst, src, count, offset);
  return cudaGetLastError();
}

cudaError_t setup_long_rows(const int* ptr, int nrows, int thresh, int* flags, int* pos, int* bsum,
                            int* list, int* h_count, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  k_long_flags<<<grid_for(nrows, G), kBlock, 0, s>>>(ptr, nrows, thresh, flags);
  RET(cudaGetLastError());
  RET(exclusive_scan(flags, pos, nrows, bsum, s));
  k_long_scatter<<<grid_for(nrows, G), kBlock, 0, s>>>(flags, pos, nrows, list);
  RET(cudaGetLastError());
  RET(cudaMemcpyAsync(h_count, pos + nrows, sizeof(int), cudaMemcpyDeviceToHost, s));
  return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------ tile items
namespace {

// cnt[r] = work items that start at row r (0: row r continues the tile before it);
// lfl[r] = 1 if row r is long.  A row starts an item if it is the first row, a
// multiple of kTileRows, long, follows a long row, or starts in another window of
// W nonzeros than the row before it.
__global__ void k_tile_count(const int* ptr, int R, int W, int rows, int* cnt, int* lfl) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += stride) {
    const int r = (int)i;
    const int s = ptr[r], e = ptr[r + 1];
    const bool lng = e - s > kLongRow;
    bool start = r == 0 || r % rows == 0 || lng;
    if (!start) {
      const int sp = ptr[r - 1];
      start = s / W != sp / W || s - sp > kLongRow;
    }
    cnt[r] = start ? (lng ? (e - s + W - 1) / W : 1) : 0;
    lfl[r] = lng ? 1 : 0;
  }
}

// the first row of every LP of a batch starts an item
__global__ void k_tile_lp_starts(const int* lp_row0, int count, int R, int* cnt) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    const int r = lp_row0[k];
    if (r < R && cnt[r] == 0) cnt[r] = 1;
  }
}

__device__ int lp_of_row(const int* lp_row0, int count, int r) {
  // the last LP whose first row is <= r (empty LPs share their first row with the next)
  int lo = 0, hi = count;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (lp_row0[mid] <= r) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_tile_emit(const int* ptr, int R, int W, const int* lp_row0, int count,
                            const int* cnt, const int* off, const int* loff, TileItem* items) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += stride) {
    const int r = (int)i;
    const int c = cnt[r];
    if (c == 0) continue;
    const int lp = lp_row0 ? lp_of_row(lp_row0, count, r) : 0;
    const int s = ptr[r], e = ptr[r + 1], i0 = off[r];
    if (e - s > kLongRow) {
      for (int t = 0; t < c; ++t)
        items[i0 + t] = TileItem{r, r + 1, s + t * W, (int)min((long long)s + (long long)(t + 1) * W,
                                                               (long long)e), lp, i0, c, loff[r]};
    } else {
      int re = r + 1;
      while (re < R && cnt[re] == 0) ++re;
      items[i0] = TileItem{r, re, s, ptr[re], lp, -1, 0, -1};
    }
  }
}

__global__ void k_tile_lp_ranges(const int* lp_row0, int count, int R, const int* off,
                                 const int* loff, int* item0, int* lng0) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= count; k += gridDim.x * blockDim.x) {
    const int r = k == count ? R : (lp_row0 ? lp_row0[k] : 0);
    item0[k] = off[r];
    lng0[k] = loff[r];
  }
}

}  // namespace

TileShape tile_shape(int form) {
  return form == 2 ? TileShape{kWarpTileRows, kWarpTileWindowMin, kWarpTileWindowMax}
                   : TileShape{kTileRows, kTileWindowMin, kTileWindowMax};
}

int tile_window(const TileShape& sh, int R, long long nnz) {
  const double avg = R > 0 ? (double)nnz / (double)R : 1.0;
  const double w = (double)sh.rows * avg;
  return (int)std::max((double)sh.wmin, std::min((double)sh.wmax, w));
}

size_t tile_item_cap(const TileShape& sh, int R, long long nnz, int count) {
  // starts: multiples of the row cap, crossings of the W-windows, the rows at and
  // after each long row, LP starts; plus the slices of the long rows (at most
  // nnz / W + one per long row); long rows number at most nnz / (kLongRow + 1)
  const size_t W = (size_t)tile_window(sh, R, nnz), Z = (size_t)nnz;
  const size_t nlong = Z / (kLongRow + 1) + 1;
  return (size_t)R / sh.rows + 2 * (Z / W + 1) + 3 * nlong + (size_t)count + 8;
}

size_t tile_tmp_ints(int R) { return 4 * ((size_t)R + 1) + scan_tmp_ints((long long)R + 1) + 8; }

cudaError_t setup_tiles(const TileShape& sh, const int* ptr, int R, long long nnz,
                        const int* lp_row0, int count, int* tmp, TileItem* items, int* item0,
                        int* lng0, int* ticket, size_t item_cap, int* h_counts, int* W_out,
                        cudaStream_t s) {
  const int W = tile_window(sh, R, nnz);
  *W_out = W;
  int* cnt = tmp;
  int* off = cnt + (R + 1);
  int* lfl = off + (R + 1);
  int* loff = lfl + (R + 1);
  int* bsum = loff + (R + 1);
  const int G = device_sm_count() * 8;
  if (R > 0) {
    k_tile_count<<<grid_for(R, G), kBlock, 0, s>>>(ptr, R, W, sh.rows, cnt, lfl);
    RET(cudaGetLastError());
    if (lp_row0 && count > 1) {
      k_tile_lp_starts<<<grid_for(count, G), kBlock, 0, s>>>(lp_row0, count, R, cnt);
      RET(cudaGetLastError());
    }
  }
  RET(exclusive_scan(cnt, off, R, bsum, s));
  RET(exclusive_scan(lfl, loff, R, bsum, s));
  RET(cudaMemcpyAsync(h_counts, off + R, sizeof(int), cudaMemcpyDeviceToHost, s));
  RET(cudaMemcpyAsync(h_counts + 1, loff + R, sizeof(int), cudaMemcpyDeviceToHost, s));
  RET(cudaStreamSynchronize(s));
  if ((size_t)h_counts[0] > item_cap) return cudaErrorInvalidValue;
  if (R > 0) {
    k_tile_emit<<<grid_for(R, G), kBlock, 0, s>>>(ptr, R, W, lp_row0, count, cnt, off, loff, items);
    RET(cudaGetLastError());
  }
  k_tile_lp_ranges<<<grid_for(count + 1, G), kBlock, 0, s>>>(lp_row0, count, R, off, loff, item0,
                                                              lng0);
  RET(cudaGetLastError());
  if (h_counts[0] > 0) RET(cudaMemsetAsync(ticket, 0, sizeof(int) * (size_t)h_counts[0], s));
  return cudaSuccess;
}

// ------------------------------------------------------------------ batches
namespace {

// One LP of a batch: its arrays (device) and its first global row, column and
// nonzero in the block-diagonal problem.
__global__ void k_batch_ingest(const BatchLp* lps, int64_t* rp_g, int* col_g, double* val_g,
                               double* b_g, char* sense_g, double* c_g, double* l_g, double* u_g,
                               int* err) {
  const BatchLp L = lps[blockIdx.y];
  const int k = blockIdx.y;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int e = 0;
  for (long long i = t0; i <= L.m; i += stride) {
    const int64_t v = L.rp[i];
    if (i < L.m) {
      const int64_t w = L.rp[i + 1];
      if (v < 0 || w < v || w > L.nnz) e |= ERR_ROWPTR;
      const char sn = L.sense[i];
      if (sn != 'L' && sn != 'G' && sn != 'E') e |= ERR_SENSE;
      const double bi = L.b[i];
      if (!isfinite(bi)) e |= ERR_NONFINITE;
      b_g[L.R + i] = bi;
      sense_g[L.R + i] = sn;
    }
    if ((i == 0 && v != 0) || (i == L.m && v != L.nnz)) e |= ERR_ROWPTR;
    rp_g[L.R + i] = L.Z + v;  // the next LP writes the same value at its first row
  }
  for (long long p = t0; p < L.nnz; p += stride) {
    const int j = L.col[p];
    const double v = L.val[p];
    if (j < 0 || j >= L.n) e |= ERR_COL;
    if (!isfinite(v)) e |= ERR_NONFINITE;
    col_g[L.Z + p] = (int)L.C + j;
    val_g[L.Z + p] = v;
  }
  for (long long j = t0; j < L.n; j += stride) {
    const double cj = L.c[j], lj = L.l[j], uj = L.u[j];
    if (!isfinite(cj)) e |= ERR_NONFINITE;
    if (isnan(lj) || isnan(uj) || lj > uj || lj == INFINITY || uj == -INFINITY) e |= ERR_BOUNDS;
    c_g[L.C + j] = cj;
    l_g[L.C + j] = lj;
    u_g[L.C + j] = uj;
  }
  if (e) atomicOr(err + k, e);
}

// The A3 scalars of each LP (one block per LP), as k_iter_vectors and k_absmax_scaled
// take them for one LP: out[8 k + ...] = ||c~||, ||q~||, ||c||, ||q||, max |K~_ij|, 0, 0,
// columns with an infinite bound.
__global__ void k_batch_scalars(const BatchLp* lps, const double* dr, const double* dc,
                                const double* c, const double* l, const double* u,
                                const double* q, const int* a_ptr, const int* a_col,
                                const double* a_val64, double* out) {
  const BatchLp L = lps[blockIdx.x];
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long long j = L.C + threadIdx.x; j < L.C + L.n; j += blockDim.x) {
    const double d = dc[j], cj = c[j];
    acc[0] += (d * cj) * (d * cj);
    acc[2] += cj * cj;
    acc[6] += (isfinite(l[j]) && isfinite(u[j])) ? 0.0 : 1.0;
  }
  for (long long i = L.R + threadIdx.x; i < L.R + L.m; i += blockDim.x) {
    const double d = dr[i], qi = q[i];
    acc[1] += (d * qi) * (d * qi);
    acc[3] += qi * qi;
  }
  double mx = 0.0;
  const int lane = threadIdx.x & 31;
  for (long long r = L.R + (threadIdx.x >> 5); r < L.R + L.m; r += blockDim.x / 32) {
    const int s = a_ptr[r], e = a_ptr[r + 1];
    for (int p = s + lane; p < e; p += 32) mx = fmax(mx, fabs((dr[r] * a_val64[p]) * dc[a_col[p]]));
  }
  double r7[7];
  block_sum<7>(acc, r7);
  __shared__ double sh[kWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; ++w) mx = fmax(mx, sh[w]);
    double* o = out + 8 * (size_t)blockIdx.x;
    o[0] = sqrt(r7[0]);
    o[1] = sqrt(r7[1]);
    o[2] = sqrt(r7[2]);
    o[3] = sqrt(r7[3]);
    o[4] = mx;
    o[5] = 0.0;
    o[6] = 0.0;
    o[7] = r7[6];
  }
}

// counts[k] = entries of `pos` (an exclusive scan over global rows) before LP k's first row
__global__ void k_batch_bounds(const BatchLp* lps, int count, int over_cols, int R,
                               const int* pos, int* out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= count; k += gridDim.x * blockDim.x) {
    const long long r = k == count ? R : (over_cols ? lps[k].C : lps[k].R);
    out[k] = pos[r];
  }
}

}  // namespace

cudaError_t setup_batch_ingest(const BatchLp* d_lps, int count, long long max_rows_nnz_cols,
                               int64_t* rp_g, int* col_g, double* val_g, double* b_g,
                               char* sense_g, double* c_g, double* l_g, double* u_g, int* d_err,
                               cudaStream_t s) {
  RET(cudaMemsetAsync(d_err, 0, sizeof(int) * (size_t)count, s));
  if (count == 0) return cudaSuccess;
  const int per_lp = (int)std::min<long long>(64, std::max<long long>(1, (max_rows_nnz_cols + kBlock - 1) / kBlock));
  dim3 grid((unsigned)per_lp, (unsigned)count);
  k_batch_ingest<<<grid, kBlock, 0, s>>>(d_lps, rp_g, col_g, val_g, b_g, sense_g, c_g, l_g, u_g,
                                         d_err);
  return cudaGetLastError();
}

cudaError_t setup_batch_scalars(const BatchLp* d_lps, int count, const double* dr,
                                const double* dc, const double* c, const double* l,
                                const double* u, const double* q, const int* a_ptr,
                                const int* a_col, const double* a_val64, double* out,
                                cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  k_batch_scalars<<<count, kBlock, 0, s>>>(d_lps, dr, dc, c, l, u, q, a_ptr, a_col, a_val64, out);
  return cudaGetLastError();
}

cudaError_t setup_batch_long_rows(const int* ptr, int R, int thresh, const BatchLp* d_lps,
                                  int count, int over_cols, int* flags, int* pos, int* bsum,
                                  int* list, int* d_bounds, cudaStream_t s) {
  const int G = device_sm_count() * 8;
  if (R > 0) {
    k_long_flags<<<grid_for(R, G), kBlock, 0, s>>>(ptr, R, thresh, flags);
    RET(cudaGetLastError());
  }
  RET(exclusive_scan(flags, pos, R, bsum, s));
  if (R > 0) {
    k_long_scatter<<<grid_for(R, G), kBlock, 0, s>>>(flags, pos, R, list);
    RET(cudaGetLastError());
  }
  k_batch_bounds<<<grid_for(count + 1, G), kBlock, 0, s>>>(d_lps, count, over_cols, R, pos,
                                                            d_bounds);
  return cudaGetLastError();
}

}  // namespace pdlp
