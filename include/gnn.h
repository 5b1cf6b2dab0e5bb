/*
 * gnn.h -- C ABI of the learned warm start of the GB300 PDLP library.
 *
 * The paper starts PDLP cold (x = proj(0), y = 0) on every LP relaxation it
 * fixes from (Kempke & Koch, section 2 and section 4, "Hardware and
 * software").  This part adds a learned start: a small message-passing network
 * over the bipartite variable / constraint graph of A predicts (x0, y0), the
 * prediction is projected onto the bounds and the dual cone, and PDLP starts
 * from it only if its relative KKT error (the measure of pdlp.h, section 4's
 * relative tolerances) is below that of the cold start -- cold PDLP stays the
 * fallback and decides which start is taken.  The network is not in the paper; its definition:
 *
 *   hidden width H = 64, L = 3 layers, weights stored in bfloat16 (float32
 *   master copies for training), all arithmetic in float32;
 *   features  F_v[j] = (c_j / max|c|, g(l_j), g(u_j), ||A_:j||_2 / max_j, deg_j / max_j, 1),
 *             g(v) = sign(v) log(1 + |v|) of v clipped to [-1e3, 1e3];
 *             F_c[i] = (b_i / max|b|, s_i, ||A_i:||_2 / max_i, deg_i / max_i, 1),
 *             s_i = +1 on 'G' rows, -1 on 'L' rows, 0 on 'E' rows;
 *   embed     H_v0 = relu(F_v W_vin + b_vin),  H_c0 = relu(F_c W_cin + b_cin);
 *   layer k   S_c = R H_v(k),   R_ij = a_ij / deg_i   (mean over a row's columns),
 *             H_c(k+1) = relu(H_c(k) W_cc_k + S_c W_cv_k + b_c_k),
 *             S_v = C^T H_c(k+1),   C_ij = a_ij / deg_j (mean over a column's rows),
 *             H_v(k+1) = relu(H_v(k) W_vv_k + S_v W_vc_k + b_v_k);
 *   heads     z_x = H_v3 w_x + b_x,  x^ = l + (u - l) sigmoid(z_x) on finite boxes, else z_x;
 *             z_y = H_c3 w_y + b_y,  y^ = softplus(z_y) on inequality rows, z_y on '=' rows;
 *             the dual prediction is in units of max|c| and in the >=-form sign
 *             convention; outputs are returned in the caller's convention of pdlp.h;
 *   loss      mean_j ((x^_j - x*_j) / (u_j - l_j))^2 + mean_i (y^_i - y*_i / max|c|)^2,
 *             (u_j - l_j) replaced by 1 where the box is infinite or empty;
 *   training  Adam (Kingma & Ba 2015) on the float32 masters, bias-corrected,
 *             the bfloat16 copy refreshed after every step.
 * Parameters are one flat float32 vector in this order (W row-major [in][out]):
 *   W_vin[6][64] b_vin[64] W_cin[5][64] b_cin[64], then per layer k = 0..2
 *   W_cc_k[64][64] W_cv_k[64][64] b_c_k[64] W_vv_k[64][64] W_vc_k[64][64] b_v_k[64],
 *   then w_x[64] b_x[1] w_y[64] b_y[1]  -- gnn_param_count() = 50498 values.
 *
 * Conventions: LP data as in pdlp.h (CSR with int64 row_ptr, senses 'L'/'G'/'E',
 * +-INFINITY bounds), all pointers HOST unless stated; return codes are
 * PDLP_OK or PDLP_ERR_* of pdlp.h; pdlp_last_error() names the cause.  A model
 * and the graphs used with it live on the CUDA device that was current when
 * the model was created, and run on the model's own stream; a model is not
 * safe to use from two host threads at once.
 */
#ifndef PDLP_GNN_H
#define PDLP_GNN_H

#include <stddef.h>
#include <stdint.h>

#include "pdlp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GNN_HIDDEN 64
#define GNN_LAYERS 3
#define GNN_VAR_FEATURES 6
#define GNN_CON_FEATURES 5

typedef struct gnn_model gnn_model; /* opaque: parameters, optimiser state, scratch */
typedef struct gnn_graph gnn_graph; /* opaque: one LP's graph, features, optional labels */

/* Number of float32 parameters (50498). */
int64_t gnn_param_count(void);

/* New model on the current device: W blocks and w_x, w_y Xavier-uniform,
 * (2 U - 1) sqrt(6 / (fan_in + fan_out)) with fan (in, out) of the block
 * (w_x, w_y: (64, 1)), U the SplitMix64 uniform (r >> 11) 2^-53 of `seed`
 * drawn block by block in parameter order, each value rounded to float32;
 * biases 0; Adam moments 0, step counter 0.  *out receives the handle. */
int gnn_create(uint64_t seed, gnn_model** out);
/* Frees the model and its device memory (NULL is a no-op). */
int gnn_free(gnn_model* m);

/* Copy the float32 master parameters out ([gnn_param_count()]) or in; setting
 * them refreshes the bfloat16 copy (round to nearest, ties to even) and keeps
 * the Adam state. */
int gnn_get_params(const gnn_model* m, float* out);
int gnn_set_params(gnn_model* m, const float* in);
/* Accumulated gradient (float32, [gnn_param_count()]): read, overwrite, zero. */
int gnn_get_grad(const gnn_model* m, float* out);
int gnn_set_grad(gnn_model* m, const float* in);
int gnn_zero_grad(gnn_model* m);

/* Save / load the parameters and the Adam state to / from a file (a small
 * binary format: magic "PDLPGNN1", count, step, then params, m, v). */
int gnn_save(const gnn_model* m, const char* path);
int gnn_load(const char* path, gnn_model** out);

/* Build the graph of an LP on the model's device (inputs as in pdlp_solve):
 * validates the LP, copies A, builds the transpose and both feature matrices
 * (the features kernel).  Optional labels are set separately. */
int gnn_graph_create(gnn_model* m, const pdlp_csr* A, const double* b, const char* sense,
                     const double* c, const double* l, const double* u, gnn_graph** out);
/* Training targets: a solution x_star[n] and its duals y_star[m] in the
 * caller's convention of pdlp.h (flipped to the >=-form internally). */
int gnn_graph_set_labels(gnn_graph* g, const double* x_star, const double* y_star);
/* Feature matrices as built, row-major float32: fv[n][6], fc[m][5] (either NULL). */
int gnn_graph_features(const gnn_graph* g, float* fv, float* fc);
int gnn_graph_free(gnn_graph* g);

/* Forward pass: x_out[n], y_out[m] (float64 copies of the float32 predictions,
 * caller's sign convention; either may be NULL).  loss (may be NULL) receives
 * the loss when the graph has labels, else NaN. */
int gnn_forward(gnn_model* m, gnn_graph* g, double* x_out, double* y_out, double* loss);
/* Forward and backward pass: adds scale * dloss/dtheta to the accumulated
 * gradient (derivatives with respect to the bfloat16 weights the forward pass
 * used); loss (may be NULL) receives the loss.  Needs labels. */
int gnn_backward(gnn_model* m, gnn_graph* g, double scale, double* loss);

typedef struct {
  size_t struct_size; /* sizeof(gnn_adam); set by gnn_default_adam */
  double lr;          /* 1e-3 */
  double beta1;       /* 0.9 */
  double beta2;       /* 0.999 */
  double eps;         /* 1e-8 */
} gnn_adam;
int gnn_default_adam(gnn_adam* a);
/* One Adam step with the accumulated gradient (the step counter advances first). */
int gnn_adam_step(gnn_model* m, const gnn_adam* a);

typedef struct {
  size_t struct_size; /* sizeof(gnn_train_params); set by gnn_default_train */
  int epochs;         /* passes over the graphs, default 30 */
  int batch;          /* graphs per Adam step (gradient averaged), default 4 */
  gnn_adam adam;      /* optimiser settings */
  double lr_decay;    /* learning rate multiplied by this after every epoch, default 0.95 */
  uint64_t seed;      /* SplitMix64 seed of the per-epoch shuffle, default 1 */
} gnn_train_params;
int gnn_default_train(gnn_train_params* t);
/* Train on `count` labelled graphs: every epoch visits the graphs in a
 * Fisher-Yates order drawn from the seed, averages the gradient over `batch`
 * graphs and takes an Adam step.  epoch_loss[epochs] (may be NULL) receives
 * each epoch's mean loss.  Runs on the device; returns after the last step. */
int gnn_train(gnn_model* m, gnn_graph* const* graphs, int count, const gnn_train_params* t,
              double* epoch_loss);

/* Relative KKT of a candidate start (x0, y0), each projected first onto
 * [l, u] and the dual cone of the caller's convention, evaluated in float64 on
 * the original data with the measures of pdlp.h.  kkt_out[4] receives
 * (rel_primal_res, rel_dual_res, rel_gap, rel_kkt).  Host inputs. */
int pdlp_start_kkt(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                   const double* l, const double* u, const double* x0, const double* y0,
                   double* kkt_out);

typedef struct {
  int used_warm;        /* 1: PDLP started from the prediction; 0: cold start */
  double warm_rel_kkt;  /* relative KKT of the projected prediction */
  double cold_rel_kkt;  /* relative KKT of the cold start (proj(0), 0) */
  double predict_s;     /* graph build + forward pass + start KKT, seconds */
} gnn_warm_info;

/* pdlp_solve with a learned start: builds the LP's graph, predicts (x0, y0),
 * projects it, compares its relative KKT with the cold start's and runs PDLP
 * from the better point (ties: cold).  The initial primal weight comes from the
 * projected prediction in either case, as in pdlp_solve_hinted (the ratio of
 * its scaled dual and primal norms, the balance the weight stands for), unless
 * p->fixed_omega > 0.  Arguments as in pdlp_solve; info (may be NULL) reports
 * the decision.  model NULL = plain cold pdlp_solve. */
int pdlp_solve_warm(gnn_model* model, const pdlp_csr* A, const double* b, const char* sense,
                    const double* c, const double* l, const double* u, const pdlp_params* p,
                    double* x_out, double* y_out, pdlp_result* r, gnn_warm_info* info);

#ifdef __cplusplus
}
#endif

#endif /* PDLP_GNN_H */
