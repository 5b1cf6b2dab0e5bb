// Host-side interfaces between the translation units of the PDLP library.
// The solver driver fills these untyped launch descriptions; each kernel
// translation unit casts them to its own element types.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "../../include/pdlp.h"

namespace pdlp {

enum Mode { MODE_FP64 = 0, MODE_FP32 = 1, MODE_BF16 = 2, MODE_PAT = 3 };

// Byte offsets of the one-block shared-memory step kernel's copy of an LP
// (smem_kernels.cuh; 16-byte aligned, -1: absent); bytes = 0: the kernel is not used.
struct SmemLayout {
  int t_ptr, t_col, t_val, a_ptr, a_col, a_val;
  int c, l, u, tw, q, sw, kind, x0, x1, y0, y1, sx, sy;
  int ot, oa;  // the columns and the rows in the order the threads take them
  int bytes;
};

// Shared memory the kernel needs for an LP of m rows, n columns and nnz nonzeros with
// iterate elements of `it` bytes; `vals`: the values are stored (not a 0/1 pattern);
// `implicit`: the per-element step weights tw / sw are kept.  bytes saturates at 2^30.
inline SmemLayout smem_layout(long long m, long long n, long long nnz, int it, bool vals,
                              bool implicit) {
  SmemLayout L;
  long long o = 0;
  auto take = [&o](long long b) -> int {
    const long long r = o;
    o += (b + 15) / 16 * 16;
    return (int)(r < (1LL << 30) ? r : (1LL << 30));
  };
  L.t_ptr = take(4 * (n + 1));
  L.t_col = take(4 * nnz);
  L.t_val = vals ? take(it * nnz) : -1;
  L.a_ptr = take(4 * (m + 1));
  L.a_col = take(4 * nnz);
  L.a_val = vals ? take(it * nnz) : -1;
  L.c = take(it * n);
  L.l = take(it * n);
  L.u = take(it * n);
  L.tw = implicit ? take(it * n) : -1;
  L.q = take(it * m);
  L.sw = implicit ? take(it * m) : -1;
  L.kind = take(m);
  L.x0 = take(2 * it * n);
  L.x1 = take(2 * it * n);
  L.y0 = take(it * m);
  L.y1 = take(it * m);
  L.sx = take(it * n);
  L.sy = take(it * m);
  L.ot = take(4 * n);
  L.oa = take(4 * m);
  L.bytes = (int)(o < (1LL << 30) ? o : (1LL << 30));
  return L;
}

struct IterRaw {
  const int *a_ptr, *a_col;
  const void* a_val;
  const int *t_ptr, *t_col;
  const void* t_val;
  const int *a_long, *t_long;
  int a_nlong, t_nlong, a_thresh, t_thresh;
  int m, n;
  const void *c, *l, *u, *q, *tw, *sw;
  const unsigned char* row_kind;
  void *x[2], *y[2], *sum_x, *sum_y;  // x: interleaved (x_j, dx_j) pairs
  double *part_p, *part_d;
  int grid_p_short, grid_p, grid_d_short, grid_d;
  DevState* st;  // [count]
  int count;     // LPs (1 for a single LP)
  unsigned long long cond;  // while-loop handle of the check-period graph (0: none)
  int loop_cap;             // attempts per graph launch at most (with cond)
  Tables tp, td; // batch tables over A^T and A (all NULL for one LP)
  // tile step kernels (float32 iterates): 0 off, 1 staged block tiles
  // (tile_kernels.cuh), 2 warp tiles (wtile_kernels.cuh)
  int tile;
  TileSet tt, ta;        // items over A^T (primal step) and over A (dual step)
  int grid_tt, grid_ta;  // their grids (blocks)
  int work_tt, work_ta;  // workers (blocks or warps): k_decide reads one slot per worker and LP
  int tslot;             // partials per slot (8 for block tiles, 1 for warp tiles)
  // one-block persistent form (persistent = 2): smem.bytes > 0 runs k_smem, the LP held in
  // that much shared memory; 0 runs the one-block k_persist from global memory
  SmemLayout smem;
  const int *ord_t, *ord_a;  // its order of the columns and rows (longest first)
  // Halpern variant (pdlp_params.halpern): its iterate and anchor (iterate type; NULL off)
  void *hx, *hy;
  const void *hax, *hay;
};

// IK_DUAL launches the dual step kernel and then the step decision (k_decide)
enum IterKernel { IK_PRIMAL = 0, IK_DUAL = 1 };

// persistent attempts kernel (one LP; see iter_kernels.cuh): grid 0 = resident maximum
cudaError_t launch_persist_fp64(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                                int grid, int* grid_out, cudaStream_t s);
cudaError_t launch_persist_fp32(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                                int grid, int* grid_out, cudaStream_t s);
cudaError_t launch_persist_bf16(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                                int grid, int* grid_out, cudaStream_t s);
cudaError_t launch_persist_pat(int lanes_a, int lanes_t, const IterRaw& r, int max_attempts,
                               int grid, int* grid_out, cudaStream_t s);

// blocks of the tile kernels of a form (primal, dual) resident at once on this device
cudaError_t tile_resident_fp32(int form, int* primal_blocks, int* dual_blocks);
cudaError_t tile_resident_bf16(int form, int* primal_blocks, int* dual_blocks);
cudaError_t tile_resident_pat(int form, int* primal_blocks, int* dual_blocks);

cudaError_t launch_iter_fp64(int which, int lanes, const IterRaw& r, cudaStream_t s);
cudaError_t launch_iter_fp32(int which, int lanes, const IterRaw& r, cudaStream_t s);
cudaError_t launch_iter_bf16(int which, int lanes, const IterRaw& r, cudaStream_t s);
cudaError_t launch_iter_pat(int which, int lanes, const IterRaw& r, cudaStream_t s);
// the Halpern variant's step kernels (two launches per attempt only)
cudaError_t launch_iter_fp64_h(int which, int lanes, const IterRaw& r, cudaStream_t s);
cudaError_t launch_iter_fp32_h(int which, int lanes, const IterRaw& r, cudaStream_t s);
cudaError_t launch_iter_bf16_h(int which, int lanes, const IterRaw& r, cudaStream_t s);
cudaError_t launch_iter_pat_h(int which, int lanes, const IterRaw& r, cudaStream_t s);

struct KktRaw {
  const int *a_ptr, *a_col;
  const double* a_val64;  // raw canonical K (NULL: every value is +1, the pattern mode)
  const int *t_ptr, *t_col;
  const double* t_val64;
  const int *a_long, *t_long;
  int a_nlong, t_nlong, a_thresh, t_thresh;
  int m, n;
  const double *c, *l, *u, *q, *dr, *dc;  // unscaled canonical data, scaling
  const double *inv_dr, *inv_dc;           // 1 / D_r, 1 / D_c
  const unsigned char* bflags;             // per column: bit 0 l finite, bit 1 u finite
  const unsigned char* row_kind;           // 0 >=-row, 1 =-row, 2 <=-row flipped to >=
  void *x[2], *y[2], *sum_x, *sum_y;       // iterates (float or double; x as (x_j, dx_j) pairs)
  // the float64 candidates of each column / row of a KKT check, unscaled:
  // (current, average) side by side, so a gathered entry is one 16-byte load; the
  // certificate rays x - x_last, y - y_last (projected onto the recession cone of
  // [l, u] and onto Y) in arrays of their own, written and read only when the
  // certificate test needs them (XR with rays = 2, YR with rays >= 1)
  double2 *XG, *YG;
  double *XR, *YR;
  double *Xl, *Yl;  // unscaled restart anchors
  // Halpern variant: its iterate and anchor (iterate type), reset to the candidate at a
  // restart (NULL off)
  void *hx, *hy, *hax, *hay;
  // normalized-duality-gap restarts (NULL off): the scaled gap gradients premultiplied by
  // D_c (columns) and D_r (rows) for (current, average), written by the KKT passes; the
  // bisection state; 4 partials per block of k_ndg_eval (grid_e blocks)
  double2 *ndg_gx, *ndg_gy;
  NdgState* ndg;
  double* ndg_part;
  double* chk_pts;  // [chk_cap x n] current point of the last checks (NULL: not kept)
  long long chk_cap;
  double *part_r, *part_c;                 // kPartR / kPartC partial rows of grid_r / grid_c
  int rays;  // ray terms in the KKT passes: 0 none, 1 the dual ray only (every column
             // boxed, so the primal ray is 0), 2 both
  int grid_r_short, grid_r, grid_c_short, grid_c, grid_e;
  int scaled;  // iterates are in scaled space (explicit K~)
  // iterates in unscaled space (scaled = 0): the factors that carry them to the original
  // units, beta and gamma of the bound-objective rescaling (1 without it); in scaled space
  // the factors are folded into dc and dr
  double ux, uy;
  int fp32;    // iterate element type is float
  DevState* st;  // [count]
  int count;     // LPs in the batch (1 for a single LP)
  Tables tr, tc; // batch tables over A and A^T (all NULL for one LP); the elementwise
                 // kernels use tc's block map with grid_c blocks
};

// partial sums per block of the KKT passes over A (rows) and A^T (columns)
constexpr int kPartR = 11;
constexpr int kPartC = 15;

enum KktKernel { KK_PREP = 0, KK_ROWS = 1, KK_COLS = 2, KK_FINAL = 3, KK_APPLY = 4, KK_END = 5,
                 KK_NDG = 6, KK_NDG_BLOCK = 7 };
cudaError_t launch_kkt(int which, int lanes_r, int lanes_c, const KktRaw& r, cudaStream_t s);
// Final outputs in the caller's convention: x clipped to [l,u], y sign-flipped
// back on <=-rows.  Any pointer may be NULL.
cudaError_t launch_output(const KktRaw& r, double* x_out, double* y_out, double* x_cur,
                          double* y_cur, double* x_avg, double* y_avg, cudaStream_t s);

// pdlp_solve_device (device buffers, stream order) whose initial primal weight is
// ||y~_h|| / ||x~_h|| of the hint (hx, hy), projected and scaled like a start
int solve_device_hint(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                      const double* l, const double* u, const pdlp_params* p, const double* x0,
                      const double* y0, const double* hx, const double* hy, double* x_out,
                      double* y_out, pdlp_result* r, cudaStream_t s);

int grid_for(long long work_items, int max_blocks);

// Launch of a kernel of the iteration chain with programmatic dependent launch
// (the kernel calls pdl_enter() first).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}
// the same with `smem` bytes of dynamic shared memory
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), int grid, int block, int smem, cudaStream_t s,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}
int device_sm_count();

}  // namespace pdlp
