// Host interfaces of the device setup (validation, canonical form, transpose,
// scaling, iteration-space data).
#pragma once

#include "internal.h"

namespace pdlp {

enum SetupError { ERR_ROWPTR = 1, ERR_COL = 2, ERR_NONFINITE = 4, ERR_SENSE = 8, ERR_BOUNDS = 16 };

struct SetupIn {  // caller's arrays (device)
  int m, n;
  long long nnz;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double *b;
  const char* sense;
  const double *c, *l, *u;
};

struct ScaleIn {
  int m, n;
  const int *a_ptr, *a_col;
  const double* a_val64;
  const int *t_ptr, *t_col;
  const double* t_val64;
  int ruiz_iters;
  double pc_alpha;  // < 0: no Pock-Chambolle pass
  long long nnz;    // nonzeros (picks the lanes per row of the statistics passes)
};

struct VecIn {
  int m, n;
  const double *dr, *dc;
  const double *c, *l, *u, *q;  // canonical float64 data
  const unsigned char* row_kind;
  const double *x0, *y0;        // caller warm start (device) or NULL
  int scaled;
  const double *wx, *wy;        // primal-weight hint (device, caller convention) or NULL
};

cudaError_t setup_validate(const SetupIn& in, int* d_err, cudaStream_t s);
cudaError_t setup_canonical(const SetupIn& in, int* a_ptr, int* a_col, double* a_val64, double* q,
                            unsigned char* row_kind, cudaStream_t s);
size_t transpose_tmp_ints(int m, int n, long long nnz);
// device_desc: build the long-segment tile descriptors on the device instead of
// in host vectors (no host allocation)
cudaError_t setup_transpose(int m, int n, int nnz, const int* a_ptr, const int* a_col,
                            const double* a_val64, int* t_ptr, int* t_col, double* t_val64,
                            int* tmp, cudaStream_t s, bool device_desc = false);
cudaError_t setup_scaling(const ScaleIn& sc, double* dr, double* dc, double* stat_r,
                          double* stat_c, cudaStream_t s);
cudaError_t setup_value_format(const double* val64, int nnz, int* d_flags, int* h_bf16_exact,
                               int* h_all_one, cudaStream_t s);
// which_type: 0 double, 1 float, 2 bfloat16
cudaError_t setup_iter_values(int which_type, const int* ptr, const int* col, const double* val64,
                              int nrows, const double* own, const double* other, int own_is_row,
                              int scaled, void* out, cudaStream_t s);
size_t setup_part_doubles(int m, int n);
// scalars_out: [0] ||c~||, [1] ||q~||, [2] ||c||, [3] ||q||, [4] max |K~_ij|,
// [5] ||x~_hint||, [6] ||y~_hint|| (scaled space, projected; 0 without a hint),
// [7] the number of columns with an infinite bound
cudaError_t setup_iter_vectors(const VecIn& v, int fp32, void* c, void* l, void* u, void* q,
                               void* tw, void* sw, void* x0, void* y0, const int* a_ptr,
                               const int* a_col, const double* a_val64, double* part,
                               double* scalars_out, cudaStream_t s);
size_t scan_tmp_ints(long long N);
// dst[i] = src[i] + offset (index arrays moved into a batch's global numbering)
cudaError_t setup_offset_copy(int* dst, const int* src, long long count, int offset,
                              cudaStream_t s);
// The rows of a CSR matrix by descending length, ties by index (ord[place] = row).
cudaError_t setup_len_order(const int* ptr, int rows, int* ord, cudaStream_t s);
// Halpern variant: the matrix of the power iteration, A and A^T in CSR (values NULL:
// every entry +1) with their long-row lists (rows longer than the thresholds, one block
// each) and the scalings D_r, D_c.
struct PowIn {
  const int *a_ptr, *a_col;
  const double* a_val;
  const int *t_ptr, *t_col;
  const double* t_val;
  const int *a_long, *t_long;
  int a_nlong, t_nlong, a_thresh, t_thresh;
  int m, n;
  const double *dr, *dc;
};
// *L = the power-iteration estimate of ||D_r K D_c||_2 after `iters` passes from
// v = 1/sqrt(n); u[m], w[n], part[part_cap] and s_dev[1] are scratch; synchronises the
// stream to read the result; *launches grows by the kernels launched.
cudaError_t setup_power_norm(const PowIn& q, int iters, double* u, double* w, double* part,
                             int part_cap, double* s_dev, double* L, long long* launches,
                             cudaStream_t s);

// Bound-objective rescaling of the iteration vectors and the start point, with the
// factors beta (right-hand side, bounds, x) and gamma (objective, y) folded into the
// KKT passes' D_r, D_c and their inverses (k_rescale in setup.cu).
cudaError_t setup_rescale(int m, int n, int fp32, double beta, double gamma, void* c, void* l,
                          void* u, void* q, void* x0, void* y0, double* dr, double* dc,
                          double* inv_dr, double* inv_dc, cudaStream_t s);
cudaError_t setup_kkt_aux(int m, int n, const double* dr, const double* dc, const double* l,
                          const double* u, double* inv_dr, double* inv_dc, unsigned char* bflags,
                          cudaStream_t s);
cudaError_t setup_long_rows(const int* ptr, int nrows, int thresh, int* flags, int* pos, int* bsum,
                            int* list, int* h_count, cudaStream_t s);

// Work items of the staged tile step kernels over one orientation of a matrix with
// R rows (int32 row pointers ptr[R + 1], global numbering for a batch): items[],
// per-LP first item item0[count + 1] and first long-row slot lng0[count + 1]
// (lp_row0[count]: each LP's first row, NULL for one LP), tickets zeroed.
// h_counts[0] = items, h_counts[1] = long rows (read back; the stream is
// synchronised).  cudaErrorInvalidValue if the items exceed item_cap.
// form 1: the staged block tiles; form 2: warp tiles
struct TileShape {
  int rows, wmin, wmax;  // rows of an item at most; range of the window W
};
TileShape tile_shape(int form);
int tile_window(const TileShape& sh, int R, long long nnz);
size_t tile_item_cap(const TileShape& sh, int R, long long nnz, int count);
size_t tile_tmp_ints(int R);
cudaError_t setup_tiles(const TileShape& sh, const int* ptr, int R, long long nnz,
                        const int* lp_row0, int count, int* tmp, TileItem* items, int* item0,
                        int* lng0, int* ticket, size_t item_cap, int* h_counts, int* W_out,
                        cudaStream_t s);

// ---- batches: many LPs set up together as one block-diagonal problem
// One LP of a batch: its arrays (device) and its first global row, column and
// nonzero.
struct BatchLp {
  const int64_t* rp;
  const int32_t* col;
  const double* val;
  const double* b;
  const char* sense;
  const double *c, *l, *u;
  int m, n;
  long long nnz;
  long long R, C, Z;
};
// Validates every LP (error bits per LP into d_err[count]) and writes the batch in
// global numbering: int64 row pointers rp_g[M + 1], column indices shifted by each
// LP's first column, values, b, senses, c, l, u.
cudaError_t setup_batch_ingest(const BatchLp* d_lps, int count, long long max_rows_nnz_cols,
                               int64_t* rp_g, int* col_g, double* val_g, double* b_g,
                               char* sense_g, double* c_g, double* l_g, double* u_g, int* d_err,
                               cudaStream_t s);
// The A3 scalars of every LP: out[8 count] as setup_iter_vectors' scalars_out
// (hint norms 0).
cudaError_t setup_batch_scalars(const BatchLp* d_lps, int count, const double* dr,
                                const double* dc, const double* c, const double* l,
                                const double* u, const double* q, const int* a_ptr,
                                const int* a_col, const double* a_val64, double* out,
                                cudaStream_t s);
// The global list of rows longer than thresh and each LP's first entry of it
// (d_bounds[count + 1]); over_cols: the rows are the LPs' columns (A^T).
cudaError_t setup_batch_long_rows(const int* ptr, int R, int thresh, const BatchLp* d_lps,
                                  int count, int over_cols, int* flags, int* pos, int* bsum,
                                  int* list, int* d_bounds, cudaStream_t s);

}  // namespace pdlp
