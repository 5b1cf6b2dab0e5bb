// Learned warm start: the bipartite message-passing network of include/gnn.h,
// its training kernels and the start-point KKT that decides warm vs cold.
//
// Kernels (all float32 arithmetic on bfloat16 weights unless stated):
//   k_gnn_rowstats / k_gnn_colstats / k_gnn_feat_*   features of variables and constraints
//   k_gnn_embed / k_gnn_embed_bwd                    input layers and their weight gradients
//   k_gnn_spmm                                       message passing over A or A^T (16 lanes
//                                                    per row, one float4 of the 64-wide
//                                                    hidden row per lane)
//   k_gnn_dense / k_gnn_dense_bwd                    relu(X1 W1 + X2 W2 + b) on 64-row tiles
//                                                    staged in shared memory, and its
//                                                    backward (input and weight gradients)
//   k_gnn_head                                       prediction heads, loss and their gradient
//   k_gnn_reduce / k_gnn_loss                        per-block partials summed in a fixed
//                                                    order (training is deterministic)
//   k_gnn_adam                                       Adam on the float32 masters + bf16 copy
//   k_start_project / k_kkt_start_*                  projection of a start and its float64
//                                                    relative KKT on the original data
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/gnn.h"
#include "internal.h"
#include "setup.h"

namespace pdlp {
extern thread_local std::string g_last_error;
}

namespace {

using bf16 = __nv_bfloat16;
constexpr int H = GNN_HIDDEN;
constexpr int NB = 256;  // threads per block of every kernel here
constexpr int kDenseSmem = (128 * 64 + 64 * 132) * 4;
constexpr int kBwdSmem = (2 * 64 * 64 + 3 * 64 * 68) * 4;
constexpr int kDensePart = 2 * 4096 + 64;

int gfail(int code, const std::string& msg) {
  pdlp::g_last_error = msg;
  return code;
}

#define GTRY(x)                                                                         \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess)                                                              \
      return gfail(e_ == cudaErrorMemoryAllocation ? PDLP_ERR_OOM : PDLP_ERR_CUDA,      \
                   std::string(#x) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

#define RTRY(x)               \
  do {                        \
    int r_ = (x);             \
    if (r_ != PDLP_OK) return r_; \
  } while (0)

// ---------------------------------------------------------------- parameters
struct POff {
  int W_vin, b_vin, W_cin, b_cin;
  int W_cc[GNN_LAYERS], W_cv[GNN_LAYERS], b_c[GNN_LAYERS];
  int W_vv[GNN_LAYERS], W_vc[GNN_LAYERS], b_v[GNN_LAYERS];
  int w_x, b_x, w_y, b_y, total;
};

POff make_off() {
  POff o{};
  int p = 0;
  auto take = [&](int k) {
    const int r = p;
    p += k;
    return r;
  };
  o.W_vin = take(GNN_VAR_FEATURES * H);
  o.b_vin = take(H);
  o.W_cin = take(GNN_CON_FEATURES * H);
  o.b_cin = take(H);
  for (int k = 0; k < GNN_LAYERS; ++k) {
    o.W_cc[k] = take(H * H);
    o.W_cv[k] = take(H * H);
    o.b_c[k] = take(H);
    o.W_vv[k] = take(H * H);
    o.W_vc[k] = take(H * H);
    o.b_v[k] = take(H);
  }
  o.w_x = take(H);
  o.b_x = take(1);
  o.w_y = take(H);
  o.b_y = take(1);
  o.total = p;
  return o;
}
const POff kOff = make_off();

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

int sm_count() { return pdlp::device_sm_count(); }

int grid_rows(long long rows, int rows_per_block, int cap) {
  long long g = (rows + rows_per_block - 1) / rows_per_block;
  return (int)std::max<long long>(1, std::min<long long>(g, cap));
}

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

__device__ __forceinline__ float sigmoidf(float z) {
  const float e = expf(-fabsf(z));
  return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}
__device__ __forceinline__ float softplusf(float z) { return log1pf(expf(-fabsf(z))) + fmaxf(z, 0.f); }

__device__ __forceinline__ unsigned long long dbits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
__device__ __forceinline__ double slog(double v) {
  v = fmin(fmax(v, -1e3), 1e3);
  return v > 0 ? log1p(v) : (v < 0 ? -log1p(-v) : 0.0);
}

// ---------------------------------------------------------------- LP on the device
__global__ void k_ptr32(int m, const int64_t* __restrict__ p64, int* __restrict__ p32,
                        const char* __restrict__ sense, unsigned char* __restrict__ kind) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += gridDim.x * blockDim.x) {
    p32[i] = (int)p64[i];
    if (i < m) kind[i] = sense[i] == 'G' ? 0 : (sense[i] == 'E' ? 1 : 2);
  }
}

// ---------------------------------------------------------------- features (K11)
// maxes: [0] |b|, [1] ||A_i:||, [2] deg_i, [3] |c|, [4] ||A_:j||, [5] deg_j (float64 bits,
// all non-negative, so the unsigned order is the numeric order and atomicMax is exact)
__global__ void k_gnn_stats(int rows, const int* __restrict__ ptr, const double* __restrict__ val,
                            const double* __restrict__ rhs, double* __restrict__ norm,
                            float* __restrict__ inv_deg, unsigned long long* __restrict__ maxes) {
  unsigned long long m0 = 0, m1 = 0, m2 = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
    const int k0 = ptr[i], k1 = ptr[i + 1];
    double s = 0.0;
    for (int k = k0; k < k1; ++k) s += val[k] * val[k];
    const double nr = sqrt(s);
    const int deg = k1 - k0;
    norm[i] = nr;
    inv_deg[i] = (float)(1.0 / (double)max(deg, 1));
    m0 = max(m0, dbits(fabs(rhs[i])));
    m1 = max(m1, dbits(nr));
    m2 = max(m2, dbits((double)deg));
  }
  for (int o = 16; o > 0; o >>= 1) {
    m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&maxes[0], m0);
    atomicMax(&maxes[1], m1);
    atomicMax(&maxes[2], m2);
  }
}

__device__ __forceinline__ double umax(const unsigned long long* mx, int i, double floor) {
  return fmax(__longlong_as_double((long long)mx[i]), floor);
}

__global__ void k_gnn_feat_v(int n, const int* __restrict__ t_ptr, const double* __restrict__ c,
                             const double* __restrict__ l, const double* __restrict__ u,
                             const double* __restrict__ nc, const unsigned long long* __restrict__ mx,
                             float* __restrict__ fv) {
  const double cmax = umax(mx, 3, 1e-12), nmax = umax(mx, 4, 1e-12), dmax = umax(mx, 5, 1.0);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    float* f = fv + (size_t)j * GNN_VAR_FEATURES;
    f[0] = (float)(c[j] / cmax);
    f[1] = (float)slog(l[j]);
    f[2] = (float)slog(u[j]);
    f[3] = (float)(nc[j] / nmax);
    f[4] = (float)((double)(t_ptr[j + 1] - t_ptr[j]) / dmax);
    f[5] = 1.f;
  }
}

__global__ void k_gnn_feat_c(int m, const int* __restrict__ a_ptr, const double* __restrict__ b,
                             const unsigned char* __restrict__ kind, const double* __restrict__ nr,
                             const unsigned long long* __restrict__ mx, float* __restrict__ fc) {
  const double bmax = umax(mx, 0, 1e-12), nmax = umax(mx, 1, 1e-12), dmax = umax(mx, 2, 1.0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    float* f = fc + (size_t)i * GNN_CON_FEATURES;
    f[0] = (float)(b[i] / bmax);
    f[1] = kind[i] == 0 ? 1.f : (kind[i] == 2 ? -1.f : 0.f);
    f[2] = (float)(nr[i] / nmax);
    f[3] = (float)((double)(a_ptr[i + 1] - a_ptr[i]) / dmax);
    f[4] = 1.f;
  }
}

// ---------------------------------------------------------------- embedding
template <int NF>
__global__ void __launch_bounds__(NB) k_gnn_embed(int N, const float* __restrict__ F,
                                                  const bf16* __restrict__ W, const bf16* __restrict__ b,
                                                  float* __restrict__ out) {
  __shared__ float ws[NF * H + H];
  for (int i = threadIdx.x; i < NF * H; i += NB) ws[i] = bf(W[i]);
  for (int i = threadIdx.x; i < H; i += NB) ws[NF * H + i] = bf(b[i]);
  __syncthreads();
  const int q = threadIdx.x & 15;
  for (long long r = ((long long)blockIdx.x * NB + threadIdx.x) >> 4; r < N;
       r += (long long)gridDim.x * (NB / 16)) {
    float a[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = ws[NF * H + 4 * q + e];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float x = F[r * NF + f];
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] = fmaf(x, ws[f * H + 4 * q + e], a[e]);
    }
    st4(out + r * H + 4 * q,
        make_float4(fmaxf(a[0], 0.f), fmaxf(a[1], 0.f), fmaxf(a[2], 0.f), fmaxf(a[3], 0.f)));
  }
}

// partial per block: [NF][64] weight gradient, then [64] bias gradient
template <int NF>
__global__ void __launch_bounds__(NB) k_gnn_embed_bwd(int N, const float* __restrict__ F,
                                                      const float* __restrict__ H0,
                                                      const float* __restrict__ dH0,
                                                      float* __restrict__ part) {
  __shared__ float red[4][(NF + 1) * H];
  const int h = threadIdx.x & 63, rl = threadIdx.x >> 6;
  float g[NF + 1];
#pragma unroll
  for (int f = 0; f <= NF; ++f) g[f] = 0.f;
  for (long long r = (long long)blockIdx.x * 4 + rl; r < N; r += (long long)gridDim.x * 4) {
    const float d = H0[r * H + h] > 0.f ? dH0[r * H + h] : 0.f;
#pragma unroll
    for (int f = 0; f < NF; ++f) g[f] = fmaf(F[r * NF + f], d, g[f]);
    g[NF] += d;
  }
#pragma unroll
  for (int f = 0; f <= NF; ++f) red[rl][f * H + h] = g[f];
  __syncthreads();
  for (int e = threadIdx.x; e < (NF + 1) * H; e += NB)
    part[(size_t)blockIdx.x * (NF + 1) * H + e] = ((red[0][e] + red[1][e]) + red[2][e]) + red[3][e];
}

// ---------------------------------------------------------------- message passing (K12)
// out[r] (+)= srow[r] * sum_k val[k] * scol[col[k]] * X[col[k]]  (srow / scol may be NULL = 1)
__global__ void __launch_bounds__(NB) k_gnn_spmm(int rows, const int* __restrict__ ptr,
                                                 const int* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const float* __restrict__ srow,
                                                 const float* __restrict__ scol,
                                                 const float* __restrict__ X, float* __restrict__ out,
                                                 int accumulate) {
  const int q = threadIdx.x & 15;
  for (long long r = ((long long)blockIdx.x * NB + threadIdx.x) >> 4; r < rows;
       r += (long long)gridDim.x * (NB / 16)) {
    const int k0 = ptr[r], k1 = ptr[r + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int k = k0;
    for (; k + 4 <= k1; k += 4) {
      int j[4];
      float w[4];
      float4 x[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        j[t] = col[k + t];
        w[t] = (float)val[k + t];
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (scol) w[t] *= scol[j[t]];
        x[t] = ld4(X + (size_t)j[t] * H + 4 * q);
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc.x = fmaf(w[t], x[t].x, acc.x);
        acc.y = fmaf(w[t], x[t].y, acc.y);
        acc.z = fmaf(w[t], x[t].z, acc.z);
        acc.w = fmaf(w[t], x[t].w, acc.w);
      }
    }
    for (; k < k1; ++k) {
      const int jj = col[k];
      float w = (float)val[k];
      if (scol) w *= scol[jj];
      const float4 x = ld4(X + (size_t)jj * H + 4 * q);
      acc.x = fmaf(w, x.x, acc.x);
      acc.y = fmaf(w, x.y, acc.y);
      acc.z = fmaf(w, x.z, acc.z);
      acc.w = fmaf(w, x.w, acc.w);
    }
    if (srow) {
      const float s = srow[r];
      acc.x *= s;
      acc.y *= s;
      acc.z *= s;
      acc.w *= s;
    }
    float* o = out + r * H + 4 * q;
    if (accumulate) {
      const float4 p = ld4(o);
      acc.x += p.x;
      acc.y += p.y;
      acc.z += p.z;
      acc.w += p.w;
    }
    st4(o, acc);
  }
}

// ---------------------------------------------------------------- dense layers (K13)
// out = relu(X1 W1 + X2 W2 + b) for X1, X2 [N][64], W [64][64] row-major [in][out].
// A block stages both weights (as float) once and then 64-row tiles of [X1 | X2];
// thread (ty, tx) computes rows 4ty..4ty+3 x columns 4tx..4tx+3.
__global__ void __launch_bounds__(NB) k_gnn_dense(int N, const float* __restrict__ X1,
                                                  const float* __restrict__ X2,
                                                  const bf16* __restrict__ W1,
                                                  const bf16* __restrict__ W2,
                                                  const bf16* __restrict__ bias,
                                                  float* __restrict__ out) {
  extern __shared__ float4 smem4[];
  float* Ws = reinterpret_cast<float*>(smem4);  // [128][64]
  float* Xs = Ws + 128 * 64;                    // [64][132]
  for (int i = threadIdx.x; i < 64 * 64; i += NB) {
    Ws[i] = bf(W1[i]);
    Ws[64 * 64 + i] = bf(W2[i]);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float b4[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) b4[e] = bf(bias[4 * tx + e]);
  const int tiles = (N + 63) / 64;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long long row0 = (long long)t * 64;
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * 32; idx += NB) {
      const int r = idx >> 5, qq = idx & 31;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row0 + r < N)
        v = qq < 16 ? ld4(X1 + (row0 + r) * H + 4 * qq) : ld4(X2 + (row0 + r) * H + 4 * (qq - 16));
      st4(Xs + r * 132 + 4 * qq, v);
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = b4[j];
#pragma unroll 4
    for (int k4 = 0; k4 < 32; ++k4) {
      float4 xr[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xr[i] = ld4(Xs + (4 * ty + i) * 132 + 4 * k4);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) w[kk] = ld4(Ws + (4 * k4 + kk) * 64 + 4 * tx);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float xv[4] = {xr[i].x, xr[i].y, xr[i].z, xr[i].w};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          acc[i][0] = fmaf(xv[kk], w[kk].x, acc[i][0]);
          acc[i][1] = fmaf(xv[kk], w[kk].y, acc[i][1]);
          acc[i][2] = fmaf(xv[kk], w[kk].z, acc[i][2]);
          acc[i][3] = fmaf(xv[kk], w[kk].w, acc[i][3]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long r = row0 + 4 * ty + i;
      if (r < N)
        st4(out + r * H + 4 * tx, make_float4(fmaxf(acc[i][0], 0.f), fmaxf(acc[i][1], 0.f),
                                              fmaxf(acc[i][2], 0.f), fmaxf(acc[i][3], 0.f)));
    }
  }
}

// Backward of k_gnn_dense: dP = dHn * (Hn > 0); dX1 = dP W1^T; dX2 = dP W2^T;
// per-block partials of X1^T dP, X2^T dP (row-major [in][out]) and sum_r dP.
__global__ void __launch_bounds__(NB) k_gnn_dense_bwd(int N, const float* __restrict__ X1,
                                                      const float* __restrict__ X2,
                                                      const float* __restrict__ Hn,
                                                      const float* __restrict__ dHn,
                                                      const bf16* __restrict__ W1,
                                                      const bf16* __restrict__ W2,
                                                      float* __restrict__ dX1,
                                                      float* __restrict__ dX2,
                                                      float* __restrict__ part) {
  extern __shared__ float4 smem4[];
  float* Wt1 = reinterpret_cast<float*>(smem4);  // [64 out][64 in]
  float* Wt2 = Wt1 + 64 * 64;
  float* dPs = Wt2 + 64 * 64;                    // [64 rows][68]
  float* X1s = dPs + 64 * 68;
  float* X2s = X1s + 64 * 68;
  for (int i = threadIdx.x; i < 64 * 64; i += NB) {
    const int k = i >> 6, h = i & 63;  // W[k][h] -> Wt[h][k]
    Wt1[h * 64 + k] = bf(W1[i]);
    Wt2[h * 64 + k] = bf(W2[i]);
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float g1[4][4], g2[4][4], gb = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) g1[i][j] = g2[i][j] = 0.f;
  const int tiles = (N + 63) / 64;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const long long row0 = (long long)t * 64;
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * 16; idx += NB) {
      const int r = idx >> 4, qq = idx & 15;
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f), a = d, b = d;
      if (row0 + r < N) {
        const long long o = (row0 + r) * H + 4 * qq;
        const float4 hn = ld4(Hn + o);
        const float4 dh = ld4(dHn + o);
        d = make_float4(hn.x > 0.f ? dh.x : 0.f, hn.y > 0.f ? dh.y : 0.f,
                        hn.z > 0.f ? dh.z : 0.f, hn.w > 0.f ? dh.w : 0.f);
        a = ld4(X1 + o);
        b = ld4(X2 + o);
      }
      st4(dPs + r * 68 + 4 * qq, d);
      st4(X1s + r * 68 + 4 * qq, a);
      st4(X2s + r * 68 + 4 * qq, b);
    }
    __syncthreads();
    // input gradients: rows 4ty.., input columns 4tx..
    {
      float a1[4][4], a2[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) a1[i][j] = a2[i][j] = 0.f;
#pragma unroll 2
      for (int h4 = 0; h4 < 16; ++h4) {
        float4 d[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) d[i] = ld4(dPs + (4 * ty + i) * 68 + 4 * h4);
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          const float4 w1 = ld4(Wt1 + (4 * h4 + hh) * 64 + 4 * tx);
          const float4 w2 = ld4(Wt2 + (4 * h4 + hh) * 64 + 4 * tx);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float dv = hh == 0 ? d[i].x : (hh == 1 ? d[i].y : (hh == 2 ? d[i].z : d[i].w));
            a1[i][0] = fmaf(dv, w1.x, a1[i][0]);
            a1[i][1] = fmaf(dv, w1.y, a1[i][1]);
            a1[i][2] = fmaf(dv, w1.z, a1[i][2]);
            a1[i][3] = fmaf(dv, w1.w, a1[i][3]);
            a2[i][0] = fmaf(dv, w2.x, a2[i][0]);
            a2[i][1] = fmaf(dv, w2.y, a2[i][1]);
            a2[i][2] = fmaf(dv, w2.z, a2[i][2]);
            a2[i][3] = fmaf(dv, w2.w, a2[i][3]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const long long r = row0 + 4 * ty + i;
        if (r < N) {
          st4(dX1 + r * H + 4 * tx, make_float4(a1[i][0], a1[i][1], a1[i][2], a1[i][3]));
          st4(dX2 + r * H + 4 * tx, make_float4(a2[i][0], a2[i][1], a2[i][2], a2[i][3]));
        }
      }
    }
    // weight gradients: inputs 4ty.., outputs 4tx..
#pragma unroll 4
    for (int r = 0; r < 64; ++r) {
      const float4 x1 = ld4(X1s + r * 68 + 4 * ty);
      const float4 x2 = ld4(X2s + r * 68 + 4 * ty);
      const float4 d = ld4(dPs + r * 68 + 4 * tx);
      const float xa[4] = {x1.x, x1.y, x1.z, x1.w}, xb[4] = {x2.x, x2.y, x2.z, x2.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        g1[i][0] = fmaf(xa[i], d.x, g1[i][0]);
        g1[i][1] = fmaf(xa[i], d.y, g1[i][1]);
        g1[i][2] = fmaf(xa[i], d.z, g1[i][2]);
        g1[i][3] = fmaf(xa[i], d.w, g1[i][3]);
        g2[i][0] = fmaf(xb[i], d.x, g2[i][0]);
        g2[i][1] = fmaf(xb[i], d.y, g2[i][1]);
        g2[i][2] = fmaf(xb[i], d.z, g2[i][2]);
        g2[i][3] = fmaf(xb[i], d.w, g2[i][3]);
      }
    }
    if (threadIdx.x < 64)
      for (int r = 0; r < 64; ++r) gb += dPs[r * 68 + threadIdx.x];
  }
  float* p = part + (size_t)blockIdx.x * kDensePart;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    st4(p + (4 * ty + i) * 64 + 4 * tx, make_float4(g1[i][0], g1[i][1], g1[i][2], g1[i][3]));
    st4(p + 4096 + (4 * ty + i) * 64 + 4 * tx, make_float4(g2[i][0], g2[i][1], g2[i][2], g2[i][3]));
  }
  if (threadIdx.x < 64) p[8192 + threadIdx.x] = gb;
}

// ---------------------------------------------------------------- heads and loss
// One half-warp per row (lane q holds hidden units 4q..4q+3).  MODE 0: primal head
// (l + (u - l) sigmoid on finite boxes), MODE 1: dual head (softplus on inequality
// rows).  pred: float64 prediction in the caller's convention (may be NULL); with a
// label: loss terms, dz, dH = dz w (may be NULL) and partials [64 gw | gb].
template <int MODE>
__global__ void __launch_bounds__(NB) k_gnn_head(int N, const float* __restrict__ Hn,
                                                 const bf16* __restrict__ w,
                                                 const bf16* __restrict__ bconst,
                                                 const double* __restrict__ l,
                                                 const double* __restrict__ u,
                                                 const unsigned char* __restrict__ kind, double cmax,
                                                 const float* __restrict__ label, float two_over_n,
                                                 double* __restrict__ pred, float* __restrict__ dH,
                                                 float* __restrict__ part,
                                                 double* __restrict__ loss_part) {
  __shared__ float4 red[16][16];
  __shared__ float redb[16];
  __shared__ double redl[16];
  const int q = threadIdx.x & 15, hw = threadIdx.x >> 4;
  const unsigned mask = 0xffffu << (threadIdx.x & 16);
  const float4 wv = make_float4(bf(w[4 * q]), bf(w[4 * q + 1]), bf(w[4 * q + 2]), bf(w[4 * q + 3]));
  const float b0 = bf(bconst[0]);
  float4 gw = make_float4(0.f, 0.f, 0.f, 0.f);
  float gb = 0.f;
  double ls = 0.0;
  for (long long r = (long long)blockIdx.x * 16 + hw; r < N; r += (long long)gridDim.x * 16) {
    const float4 h = ld4(Hn + r * H + 4 * q);
    float z = h.x * wv.x + h.y * wv.y + h.z * wv.z + h.w * wv.w;
    z += __shfl_xor_sync(mask, z, 8, 16);
    z += __shfl_xor_sync(mask, z, 4, 16);
    z += __shfl_xor_sync(mask, z, 2, 16);
    z += __shfl_xor_sync(mask, z, 1, 16);
    z += b0;
    float p, dpdz, rng = 1.f;
    unsigned char kd = 0;
    if (MODE == 0) {
      const double lj = l[r], uj = u[r];
      if (isfinite(lj) && isfinite(uj)) {
        const float s = sigmoidf(z), width = (float)(uj - lj);
        p = (float)lj + width * s;
        dpdz = width * s * (1.f - s);
        rng = width > 0.f ? width : 1.f;
      } else {
        p = z;
        dpdz = 1.f;
      }
    } else {
      kd = kind[r];
      if (kd == 1) {
        p = z;
        dpdz = 1.f;
      } else {
        p = softplusf(z);
        dpdz = sigmoidf(z);
      }
    }
    if (pred && q == 0)
      pred[r] = MODE == 0 ? (double)p : (kd == 2 ? -cmax * (double)p : cmax * (double)p);
    if (label) {
      const float e = (p - label[r]) / rng;
      const float dz = two_over_n * e / rng * dpdz;
      if (q == 0) {
        ls += (double)e * (double)e;
        gb += dz;
      }
      gw.x = fmaf(dz, h.x, gw.x);
      gw.y = fmaf(dz, h.y, gw.y);
      gw.z = fmaf(dz, h.z, gw.z);
      gw.w = fmaf(dz, h.w, gw.w);
      if (dH) st4(dH + r * H + 4 * q, make_float4(dz * wv.x, dz * wv.y, dz * wv.z, dz * wv.w));
    }
  }
  if (!part) return;
  red[hw][q] = gw;
  if (q == 0) {
    redb[hw] = gb;
    redl[hw] = ls;
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int qq = threadIdx.x >> 2, c = threadIdx.x & 3;
    float s = 0.f;
    for (int i = 0; i < 16; ++i) {
      const float4 v = red[i][qq];
      s += c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
    }
    part[(size_t)blockIdx.x * 65 + threadIdx.x] = s;
  } else if (threadIdx.x == 64) {
    float s = 0.f;
    double sl = 0.0;
    for (int i = 0; i < 16; ++i) {
      s += redb[i];
      sl += redl[i];
    }
    part[(size_t)blockIdx.x * 65 + 64] = s;
    loss_part[blockIdx.x] = sl;
  }
}

// ---------------------------------------------------------------- reductions
struct Seg {
  int src, len, dst;
};
// grad[dst + e] += scale * sum_b part[b * stride + src + e], summed over b in order
__global__ void k_gnn_reduce(const float* __restrict__ part, int nblk, int stride, Seg s0, Seg s1,
                             Seg s2, float* __restrict__ grad, float scale) {
  const int total = s0.len + s1.len + s2.len;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    Seg s = s0;
    int i = e;
    if (i >= s0.len) {
      i -= s0.len;
      s = s1;
      if (i >= s1.len) {
        i -= s1.len;
        s = s2;
      }
    }
    double acc = 0.0;
    for (int b = 0; b < nblk; ++b) acc += (double)part[(size_t)b * stride + s.src + i];
    grad[s.dst + i] += scale * (float)acc;
  }
}

__global__ void k_gnn_loss(const double* __restrict__ lx, int nbx, double inv_n,
                           const double* __restrict__ ly, int nby, double inv_m,
                           double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sx = 0.0, sy = 0.0;
  for (int b = 0; b < nbx; ++b) sx += lx[b];
  for (int b = 0; b < nby; ++b) sy += ly[b];
  *out = sx * inv_n + sy * inv_m;
}

// ---------------------------------------------------------------- Adam (K14)
__global__ void k_gnn_adam(int P, float* __restrict__ theta, const float* __restrict__ grad,
                           float* __restrict__ m1, float* __restrict__ m2, bf16* __restrict__ w16,
                           float lr, float b1, float b2, float eps, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float m = b1 * m1[i] + (1.f - b1) * g;
    const float v = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = m;
    m2[i] = v;
    const float th = theta[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    theta[i] = th;
    w16[i] = __float2bfloat16_rn(th);
  }
}

__global__ void k_gnn_to_bf16(int P, const float* __restrict__ theta, bf16* __restrict__ w16) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16_rn(theta[i]);
}

// ---------------------------------------------------------------- start projection + KKT (K15)
// x onto [l, u]; y onto the caller's cone (<= 0 on 'L', >= 0 on 'G', free on 'E').
// A NaN component is replaced by the cold start's (proj(0) and 0).
__global__ void k_start_project(int n, int m, double* __restrict__ x, double* __restrict__ y,
                                const double* __restrict__ l, const double* __restrict__ u,
                                const unsigned char* __restrict__ kind, int cold) {
  const int tot = n + m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
    if (i < n) {
      double v = cold ? 0.0 : x[i];
      if (v != v) v = 0.0;
      x[i] = fmin(fmax(v, l[i]), u[i]);
    } else {
      const int r = i - n;
      double v = cold ? 0.0 : y[r];
      if (v != v) v = 0.0;
      y[r] = kind[r] == 2 ? fmin(v, 0.0) : (kind[r] == 0 ? fmax(v, 0.0) : v);
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one warp per row; partial per block: [sum r_p^2, sum q y (>=-form), sum q^2]
__global__ void __launch_bounds__(NB) k_kkt_start_rows(int m, const int* __restrict__ ptr,
                                                       const int* __restrict__ col,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ y,
                                                       const double* __restrict__ b,
                                                       const unsigned char* __restrict__ kind,
                                                       double* __restrict__ part) {
  __shared__ double red[NB / 32][3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long i = ((long long)blockIdx.x * NB + threadIdx.x) >> 5; i < m;
       i += (long long)gridDim.x * (NB / 32)) {
    double ax = 0.0;
    for (int k = ptr[i] + lane; k < ptr[i + 1]; k += 32) ax += val[k] * x[col[k]];
    ax = warp_sum_d(ax);
    if (lane == 0) {
      const double s = kind[i] == 2 ? -1.0 : 1.0;
      const double q = s * b[i];
      double rp = q - s * ax;
      if (kind[i] != 1) rp = fmax(rp, 0.0);
      s0 += rp * rp;
      s1 += q * (s * y[i]);
      s2 += q * q;
    }
  }
  if (lane == 0) {
    red[wid][0] = s0;
    red[wid][1] = s1;
    red[wid][2] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < NB / 32; ++w) s += red[w][threadIdx.x];
    part[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

// one warp per column; partial per block: [sum r_d^2, c^T x, sum c^2, bound terms of the dual]
__global__ void __launch_bounds__(NB) k_kkt_start_cols(int n, const int* __restrict__ ptr,
                                                       const int* __restrict__ row,
                                                       const double* __restrict__ val,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ y,
                                                       const double* __restrict__ c,
                                                       const double* __restrict__ l,
                                                       const double* __restrict__ u,
                                                       double* __restrict__ part) {
  __shared__ double red[NB / 32][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (long long j = ((long long)blockIdx.x * NB + threadIdx.x) >> 5; j < n;
       j += (long long)gridDim.x * (NB / 32)) {
    double aty = 0.0;
    for (int k = ptr[j] + lane; k < ptr[j + 1]; k += 32) aty += val[k] * y[row[k]];
    aty = warp_sum_d(aty);
    if (lane == 0) {
      const double lam = c[j] - aty;
      const double lp = fmax(lam, 0.0), lm = fmax(-lam, 0.0);
      const bool lf = isfinite(l[j]), uf = isfinite(u[j]);
      const double rd = (lf ? 0.0 : lp) + (uf ? 0.0 : lm);
      s0 += rd * rd;
      s1 += c[j] * x[j];
      s2 += c[j] * c[j];
      s3 += (lf ? l[j] * lp : 0.0) - (uf ? u[j] * lm : 0.0);
    }
  }
  if (lane == 0) {
    red[wid][0] = s0;
    red[wid][1] = s1;
    red[wid][2] = s2;
    red[wid][3] = s3;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < NB / 32; ++w) s += red[w][threadIdx.x];
    part[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
}

// out: rel_primal_res, rel_dual_res, rel_gap, rel_kkt
__global__ void k_kkt_start_final(const double* __restrict__ pr, int nbr,
                                  const double* __restrict__ pc, int nbc, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r[3] = {0, 0, 0}, cc[4] = {0, 0, 0, 0};
  for (int b = 0; b < nbr; ++b)
    for (int t = 0; t < 3; ++t) r[t] += pr[3 * b + t];
  for (int b = 0; b < nbc; ++b)
    for (int t = 0; t < 4; ++t) cc[t] += pc[4 * b + t];
  const double relp = sqrt(r[0]) / (1.0 + sqrt(r[2]));
  const double reld = sqrt(cc[0]) / (1.0 + sqrt(cc[2]));
  const double pobj = cc[1], dobj = r[1] + cc[3];
  const double relg = fabs(pobj - dobj) / (1.0 + fabs(pobj) + fabs(dobj));
  out[0] = relp;
  out[1] = reld;
  out[2] = relg;
  out[3] = fmax(relp, fmax(reld, relg));
}

// ---------------------------------------------------------------- host side
template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

struct LpDev {
  int m = 0, n = 0, nnz = 0;
  int64_t* ptr64 = nullptr;
  int *a_ptr = nullptr, *a_col = nullptr, *t_ptr = nullptr, *t_col = nullptr;
  double *a_val = nullptr, *t_val = nullptr;
  double *b = nullptr, *c = nullptr, *l = nullptr, *u = nullptr;
  char* sense = nullptr;
  unsigned char* kind = nullptr;
  // every array above lives in one allocation (one cudaMalloc and one cudaFree per LP, not
  // one each), followed by `extra` bytes the caller asked build_lp_dev for
  void* arena = nullptr;
  unsigned char* extra = nullptr;
  void release() {
    if (arena) cudaFree(arena);
    *this = LpDev{};
  }
};

// byte offsets of consecutive arrays, each 256-byte aligned
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  }
};

int check_host_lp(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                  const double* l, const double* u) {
  if (!A || !b || !sense || !c || !l || !u)
    if (!(A && A->m == 0 && c && l && u))
      return gfail(PDLP_ERR_INVALID_INPUT, "NULL LP array");
  if (A->m < 0 || A->n < 0 || A->nnz < 0 || A->nnz > 0x7fffffffLL)
    return gfail(PDLP_ERR_INVALID_INPUT, "invalid sizes");
  if (A->nnz > 0 && (!A->col || !A->val)) return gfail(PDLP_ERR_INVALID_INPUT, "NULL CSR arrays");
  if (!A->row_ptr) return gfail(PDLP_ERR_INVALID_INPUT, "NULL row_ptr");
  return PDLP_OK;
}

// Copies a host LP to the device, validates it there and builds int32 CSR of A and A^T.
int build_lp_dev(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                 const double* l, const double* u, cudaStream_t s, LpDev* d,
                 size_t extra_bytes = 0) {
  RTRY(check_host_lp(A, b, sense, c, l, u));
  const int m = A->m, n = A->n, nnz = (int)A->nnz;
  const size_t M = (size_t)m, N = (size_t)n, Z = (size_t)nnz;
  d->m = m;
  d->n = n;
  d->nnz = nnz;
  Carve cv;
  const size_t o_ptr64 = cv.take(8 * (M + 1)), o_aptr = cv.take(4 * (M + 1));
  const size_t o_acol = cv.take(4 * Z), o_aval = cv.take(8 * Z);
  const size_t o_tptr = cv.take(4 * (N + 1)), o_tcol = cv.take(4 * Z), o_tval = cv.take(8 * Z);
  const size_t o_b = cv.take(8 * M), o_c = cv.take(8 * N), o_l = cv.take(8 * N), o_u = cv.take(8 * N);
  const size_t o_sense = cv.take(M), o_kind = cv.take(M), o_err = cv.take(sizeof(int));
  const size_t o_extra = cv.take(extra_bytes);
  GTRY(cudaMalloc(&d->arena, cv.off));
  unsigned char* base = (unsigned char*)d->arena;
  d->ptr64 = (int64_t*)(base + o_ptr64);
  d->a_ptr = (int*)(base + o_aptr);
  d->a_col = (int*)(base + o_acol);
  d->a_val = (double*)(base + o_aval);
  d->t_ptr = (int*)(base + o_tptr);
  d->t_col = (int*)(base + o_tcol);
  d->t_val = (double*)(base + o_tval);
  d->b = (double*)(base + o_b);
  d->c = (double*)(base + o_c);
  d->l = (double*)(base + o_l);
  d->u = (double*)(base + o_u);
  d->sense = (char*)(base + o_sense);
  d->kind = base + o_kind;
  d->extra = extra_bytes ? base + o_extra : nullptr;
  GTRY(cudaMemcpyAsync(d->ptr64, A->row_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, s));
  if (nnz > 0) {
    GTRY(cudaMemcpyAsync(d->a_col, A->col, sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    GTRY(cudaMemcpyAsync(d->a_val, A->val, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
  }
  if (m > 0) {
    GTRY(cudaMemcpyAsync(d->b, b, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    GTRY(cudaMemcpyAsync(d->sense, sense, m, cudaMemcpyHostToDevice, s));
  }
  if (n > 0) {
    GTRY(cudaMemcpyAsync(d->c, c, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    GTRY(cudaMemcpyAsync(d->l, l, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    GTRY(cudaMemcpyAsync(d->u, u, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  }
  // the host row pointer decides every later size: check it before any kernel reads it
  if (A->row_ptr[0] != 0 || A->row_ptr[m] != A->nnz)
    return gfail(PDLP_ERR_INVALID_INPUT, "row_ptr must start at 0 and end at nnz");
  for (int i = 0; i < m; ++i)
    if (A->row_ptr[i + 1] < A->row_ptr[i])
      return gfail(PDLP_ERR_INVALID_INPUT, "row_ptr decreases at row " + std::to_string(i));
  int* d_err = (int*)(base + o_err);
  pdlp::SetupIn in{m, n, (long long)nnz, d->ptr64, d->a_col, d->a_val, d->b, d->sense,
                   d->c, d->l, d->u};
  cudaError_t e = pdlp::setup_validate(in, d_err, s);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  GTRY(e);
  if (herr) {
    std::string why;
    if (herr & pdlp::ERR_ROWPTR) why += " row_ptr";
    if (herr & pdlp::ERR_COL) why += " column index";
    if (herr & pdlp::ERR_NONFINITE) why += " non-finite value";
    if (herr & pdlp::ERR_SENSE) why += " sense";
    if (herr & pdlp::ERR_BOUNDS) why += " bounds (l > u or NaN)";
    return gfail(PDLP_ERR_INVALID_INPUT, "invalid LP:" + why);
  }
  const int G = sm_count() * 8;
  k_ptr32<<<grid_rows((long long)m + 1, NB, G), NB, 0, s>>>(m, d->ptr64, d->a_ptr, d->sense, d->kind);
  GTRY(cudaGetLastError());
  int* tmp = nullptr;
  GTRY(dalloc(&tmp, pdlp::transpose_tmp_ints(m, n, nnz)));
  e = pdlp::setup_transpose(m, n, nnz, d->a_ptr, d->a_col, d->a_val, d->t_ptr, d->t_col, d->t_val,
                            tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  GTRY(e);
  return PDLP_OK;
}

// float64 relative KKT of (x, y) (device, projected in place first unless `cold`
// builds the cold start into them); out[4] on the device
int start_kkt(const LpDev& d, double* x, double* y, int cold, double* part, double* out,
              cudaStream_t s) {
  const int G = sm_count() * 4;
  if (d.n + d.m > 0) {
    k_start_project<<<grid_rows((long long)d.n + d.m, NB, G), NB, 0, s>>>(d.n, d.m, x, y, d.l, d.u,
                                                                          d.kind, cold);
    GTRY(cudaGetLastError());
  }
  const int gr = grid_rows(d.m, NB / 32, G), gc = grid_rows(d.n, NB / 32, G);
  double* pr = part;
  double* pc = part + 3 * (size_t)G;
  if (d.m > 0) {
    k_kkt_start_rows<<<gr, NB, 0, s>>>(d.m, d.a_ptr, d.a_col, d.a_val, x, y, d.b, d.kind, pr);
    GTRY(cudaGetLastError());
  }
  if (d.n > 0) {
    k_kkt_start_cols<<<gc, NB, 0, s>>>(d.n, d.t_ptr, d.t_col, d.t_val, x, y, d.c, d.l, d.u, pc);
    GTRY(cudaGetLastError());
  }
  k_kkt_start_final<<<1, 32, 0, s>>>(pr, d.m > 0 ? gr : 0, pc, d.n > 0 ? gc : 0, out);
  GTRY(cudaGetLastError());
  return PDLP_OK;
}

size_t start_kkt_part_doubles() { return (size_t)7 * sm_count() * 4 + 8; }

}  // namespace

// ---------------------------------------------------------------- model / graph structs
struct gnn_model {
  int device = 0;
  cudaStream_t s = nullptr;
  int P = 0;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  bf16* w16 = nullptr;
  long long step = 0;
  // activation scratch, sized for the largest graph seen
  long long cap_n = -1, cap_m = -1;
  float *hv[GNN_LAYERS + 1] = {}, *hc[GNN_LAYERS + 1] = {}, *sv[GNN_LAYERS] = {},
        *sc[GNN_LAYERS] = {};
  float *dhv[2] = {}, *dhc[2] = {}, *dsv = nullptr, *dsc = nullptr;
  double *xpred = nullptr, *ypred = nullptr;
  float* part = nullptr;       // per-block gradient partials
  double* lpart = nullptr;     // per-block loss partials (x head, then y head)
  double* loss = nullptr;      // [1]
  int max_blocks = 0;
};

struct gnn_graph {
  gnn_model* owner = nullptr;
  LpDev d;
  float *inv_deg_r = nullptr, *inv_deg_c = nullptr;
  float *fv = nullptr, *fc = nullptr;
  float *x_star = nullptr, *y_star = nullptr;  // labels: x*, y* (>=-form) / max|c|
  double cmax = 1.0;
  int has_labels = 0;
};

namespace {

void free_scratch(gnn_model* md) {
  std::vector<void*> ps;
  for (int k = 0; k <= GNN_LAYERS; ++k) {
    ps.push_back(md->hv[k]);
    ps.push_back(md->hc[k]);
    md->hv[k] = md->hc[k] = nullptr;
  }
  for (int k = 0; k < GNN_LAYERS; ++k) {
    ps.push_back(md->sv[k]);
    ps.push_back(md->sc[k]);
    md->sv[k] = md->sc[k] = nullptr;
  }
  for (int k = 0; k < 2; ++k) {
    ps.push_back(md->dhv[k]);
    ps.push_back(md->dhc[k]);
    md->dhv[k] = md->dhc[k] = nullptr;
  }
  ps.push_back(md->dsv);
  ps.push_back(md->dsc);
  ps.push_back(md->xpred);
  ps.push_back(md->ypred);
  md->dsv = md->dsc = nullptr;
  md->xpred = md->ypred = nullptr;
  for (void* p : ps)
    if (p) cudaFree(p);
  md->cap_n = md->cap_m = -1;
}

int ensure_scratch(gnn_model* md, int n, int m) {
  if (n <= md->cap_n && m <= md->cap_m) return PDLP_OK;
  GTRY(cudaStreamSynchronize(md->s));
  const long long cn = std::max<long long>(n, md->cap_n), cm = std::max<long long>(m, md->cap_m);
  free_scratch(md);
  for (int k = 0; k <= GNN_LAYERS; ++k) {
    GTRY(dalloc(&md->hv[k], (size_t)cn * H));
    GTRY(dalloc(&md->hc[k], (size_t)cm * H));
  }
  for (int k = 0; k < GNN_LAYERS; ++k) {
    GTRY(dalloc(&md->sv[k], (size_t)cn * H));
    GTRY(dalloc(&md->sc[k], (size_t)cm * H));
  }
  for (int k = 0; k < 2; ++k) {
    GTRY(dalloc(&md->dhv[k], (size_t)cn * H));
    GTRY(dalloc(&md->dhc[k], (size_t)cm * H));
  }
  GTRY(dalloc(&md->dsv, (size_t)cn * H));
  GTRY(dalloc(&md->dsc, (size_t)cm * H));
  GTRY(dalloc(&md->xpred, (size_t)cn));
  GTRY(dalloc(&md->ypred, (size_t)cm));
  md->cap_n = cn;
  md->cap_m = cm;
  return PDLP_OK;
}

const bf16* W(const gnn_model* md, int off) { return md->w16 + off; }

// Forward pass over a graph: activations stay in the model's scratch.
int forward(gnn_model* md, gnn_graph* g, bool want_pred, bool with_label, bool want_dh) {
  const int n = g->d.n, m = g->d.m;
  RTRY(ensure_scratch(md, n, m));
  cudaStream_t s = md->s;
  const int Gs = sm_count() * 8, Gd = sm_count() * 3;
  if (n > 0) {
    k_gnn_embed<GNN_VAR_FEATURES><<<grid_rows((long long)n, NB / 16, Gs), NB, 0, s>>>(
        n, g->fv, W(md, kOff.W_vin), W(md, kOff.b_vin), md->hv[0]);
    GTRY(cudaGetLastError());
  }
  if (m > 0) {
    k_gnn_embed<GNN_CON_FEATURES><<<grid_rows((long long)m, NB / 16, Gs), NB, 0, s>>>(
        m, g->fc, W(md, kOff.W_cin), W(md, kOff.b_cin), md->hc[0]);
    GTRY(cudaGetLastError());
  }
  for (int k = 0; k < GNN_LAYERS; ++k) {
    if (m > 0) {
      k_gnn_spmm<<<grid_rows((long long)m, NB / 16, Gs), NB, 0, s>>>(
          m, g->d.a_ptr, g->d.a_col, g->d.a_val, g->inv_deg_r, nullptr, md->hv[k], md->sc[k], 0);
      GTRY(cudaGetLastError());
      k_gnn_dense<<<grid_rows((long long)m, 64, Gd), NB, kDenseSmem, s>>>(
          m, md->hc[k], md->sc[k], W(md, kOff.W_cc[k]), W(md, kOff.W_cv[k]), W(md, kOff.b_c[k]),
          md->hc[k + 1]);
      GTRY(cudaGetLastError());
    }
    if (n > 0) {
      k_gnn_spmm<<<grid_rows((long long)n, NB / 16, Gs), NB, 0, s>>>(
          n, g->d.t_ptr, g->d.t_col, g->d.t_val, g->inv_deg_c, nullptr, md->hc[k + 1], md->sv[k], 0);
      GTRY(cudaGetLastError());
      k_gnn_dense<<<grid_rows((long long)n, 64, Gd), NB, kDenseSmem, s>>>(
          n, md->hv[k], md->sv[k], W(md, kOff.W_vv[k]), W(md, kOff.W_vc[k]), W(md, kOff.b_v[k]),
          md->hv[k + 1]);
      GTRY(cudaGetLastError());
    }
  }
  const int gx = grid_rows((long long)n, 16, md->max_blocks);
  const int gy = grid_rows((long long)m, 16, md->max_blocks);
  if (n > 0) {
    k_gnn_head<0><<<gx, NB, 0, s>>>(n, md->hv[GNN_LAYERS], W(md, kOff.w_x), W(md, kOff.b_x),
                                    g->d.l, g->d.u, nullptr, g->cmax,
                                    with_label ? g->x_star : nullptr, 2.f / (float)n,
                                    want_pred ? md->xpred : nullptr, want_dh ? md->dhv[0] : nullptr,
                                    with_label ? md->part : nullptr, md->lpart);
    GTRY(cudaGetLastError());
  }
  if (m > 0) {
    k_gnn_head<1><<<gy, NB, 0, s>>>(m, md->hc[GNN_LAYERS], W(md, kOff.w_y), W(md, kOff.b_y),
                                    nullptr, nullptr, g->d.kind, g->cmax,
                                    with_label ? g->y_star : nullptr, 2.f / (float)m,
                                    want_pred ? md->ypred : nullptr, want_dh ? md->dhc[0] : nullptr,
                                    with_label ? md->part + (size_t)gx * 65 : nullptr,
                                    md->lpart + md->max_blocks);
    GTRY(cudaGetLastError());
  }
  if (with_label) {
    k_gnn_loss<<<1, 32, 0, s>>>(md->lpart, n > 0 ? gx : 0, n > 0 ? 1.0 / n : 0.0,
                                md->lpart + md->max_blocks, m > 0 ? gy : 0, m > 0 ? 1.0 / m : 0.0,
                                md->loss);
    GTRY(cudaGetLastError());
  }
  return PDLP_OK;
}

int reduce_into(gnn_model* md, int nblk, int stride, Seg a, Seg b, Seg c, float scale) {
  const int total = a.len + b.len + c.len;
  k_gnn_reduce<<<(total + NB - 1) / NB, NB, 0, md->s>>>(md->part, nblk, stride, a, b, c, md->grad,
                                                        scale);
  GTRY(cudaGetLastError());
  return PDLP_OK;
}

// Forward with labels, then backward; adds scale * gradient into md->grad.
int backward(gnn_model* md, gnn_graph* g, float scale) {
  const int n = g->d.n, m = g->d.m;
  RTRY(ensure_scratch(md, n, m));
  cudaStream_t s = md->s;
  const int Gs = sm_count() * 8, Gb = sm_count() * 2;
  // heads (with dH) -- their partials are reduced right after each head
  RTRY(forward(md, g, false, true, true));
  const int gx = grid_rows((long long)n, 16, md->max_blocks);
  const int gy = grid_rows((long long)m, 16, md->max_blocks);
  if (n > 0) RTRY(reduce_into(md, gx, 65, Seg{0, 64, kOff.w_x}, Seg{64, 1, kOff.b_x}, Seg{0, 0, 0}, scale));
  if (m > 0) {
    // the y head's partials sit after the x head's in md->part
    k_gnn_reduce<<<1, NB, 0, s>>>(md->part + (size_t)gx * 65, gy, 65, Seg{0, 64, kOff.w_y},
                                  Seg{64, 1, kOff.b_y}, Seg{0, 0, 0}, md->grad, scale);
    GTRY(cudaGetLastError());
  }
  int cur = 0;
  for (int k = GNN_LAYERS - 1; k >= 0; --k) {
    const int nxt = cur ^ 1;
    if (n > 0) {
      const int gb = grid_rows((long long)n, 64, Gb);
      k_gnn_dense_bwd<<<gb, NB, kBwdSmem, s>>>(n, md->hv[k], md->sv[k], md->hv[k + 1], md->dhv[cur],
                                               W(md, kOff.W_vv[k]), W(md, kOff.W_vc[k]),
                                               md->dhv[nxt], md->dsv, md->part);
      GTRY(cudaGetLastError());
      RTRY(reduce_into(md, gb, kDensePart, Seg{0, 4096, kOff.W_vv[k]}, Seg{4096, 4096, kOff.W_vc[k]},
                       Seg{8192, 64, kOff.b_v[k]}, scale));
      if (m > 0) {
        // dH_c += C dS_v, C_ij = a_ij / deg_j
        k_gnn_spmm<<<grid_rows((long long)m, NB / 16, Gs), NB, 0, s>>>(
            m, g->d.a_ptr, g->d.a_col, g->d.a_val, nullptr, g->inv_deg_c, md->dsv, md->dhc[cur], 1);
        GTRY(cudaGetLastError());
      }
    }
    if (m > 0) {
      const int gb = grid_rows((long long)m, 64, Gb);
      k_gnn_dense_bwd<<<gb, NB, kBwdSmem, s>>>(m, md->hc[k], md->sc[k], md->hc[k + 1], md->dhc[cur],
                                               W(md, kOff.W_cc[k]), W(md, kOff.W_cv[k]),
                                               md->dhc[nxt], md->dsc, md->part);
      GTRY(cudaGetLastError());
      RTRY(reduce_into(md, gb, kDensePart, Seg{0, 4096, kOff.W_cc[k]}, Seg{4096, 4096, kOff.W_cv[k]},
                       Seg{8192, 64, kOff.b_c[k]}, scale));
      if (n > 0) {
        // dH_v += R^T dS_c, R_ij = a_ij / deg_i
        k_gnn_spmm<<<grid_rows((long long)n, NB / 16, Gs), NB, 0, s>>>(
            n, g->d.t_ptr, g->d.t_col, g->d.t_val, nullptr, g->inv_deg_r, md->dsc, md->dhv[nxt], 1);
        GTRY(cudaGetLastError());
      }
    }
    cur = nxt;
  }
  if (n > 0) {
    const int ge = grid_rows((long long)n, 4, Gb);
    k_gnn_embed_bwd<GNN_VAR_FEATURES><<<ge, NB, 0, s>>>(n, g->fv, md->hv[0], md->dhv[cur], md->part);
    GTRY(cudaGetLastError());
    RTRY(reduce_into(md, ge, (GNN_VAR_FEATURES + 1) * H, Seg{0, GNN_VAR_FEATURES * H, kOff.W_vin},
                     Seg{GNN_VAR_FEATURES * H, H, kOff.b_vin}, Seg{0, 0, 0}, scale));
  }
  if (m > 0) {
    const int ge = grid_rows((long long)m, 4, Gb);
    k_gnn_embed_bwd<GNN_CON_FEATURES><<<ge, NB, 0, s>>>(m, g->fc, md->hc[0], md->dhc[cur], md->part);
    GTRY(cudaGetLastError());
    RTRY(reduce_into(md, ge, (GNN_CON_FEATURES + 1) * H, Seg{0, GNN_CON_FEATURES * H, kOff.W_cin},
                     Seg{GNN_CON_FEATURES * H, H, kOff.b_cin}, Seg{0, 0, 0}, scale));
  }
  return PDLP_OK;
}

int adam_step(gnn_model* md, const gnn_adam* a) {
  md->step += 1;
  const double bc1 = 1.0 - std::pow(a->beta1, (double)md->step);
  const double bc2 = 1.0 - std::pow(a->beta2, (double)md->step);
  k_gnn_adam<<<grid_rows(md->P, NB, sm_count() * 4), NB, 0, md->s>>>(
      md->P, md->theta, md->grad, md->m1, md->m2, md->w16, (float)a->lr, (float)a->beta1,
      (float)a->beta2, (float)a->eps, (float)bc1, (float)bc2);
  GTRY(cudaGetLastError());
  return PDLP_OK;
}

int check_model(const gnn_model* md) {
  if (!md) return gfail(PDLP_ERR_INVALID_INPUT, "NULL model");
  int dev = -1;
  GTRY(cudaGetDevice(&dev));
  if (dev != md->device)
    return gfail(PDLP_ERR_INVALID_INPUT, "the model lives on device " + std::to_string(md->device) +
                                             ", current device is " + std::to_string(dev));
  return PDLP_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" {

int64_t gnn_param_count(void) { return kOff.total; }

int gnn_create(uint64_t seed, gnn_model** out) {
  if (!out) return gfail(PDLP_ERR_INVALID_INPUT, "NULL output handle");
  *out = nullptr;
  gnn_model* md = new gnn_model();
  auto bail = [&](int code) {
    gnn_free(md);
    return code;
  };
  cudaError_t e = cudaGetDevice(&md->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&md->s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return bail(gfail(PDLP_ERR_CUDA, cudaGetErrorString(e)));
  md->P = kOff.total;
  md->max_blocks = sm_count() * 8;
  if (dalloc(&md->theta, md->P) != cudaSuccess || dalloc(&md->grad, md->P) != cudaSuccess ||
      dalloc(&md->m1, md->P) != cudaSuccess || dalloc(&md->m2, md->P) != cudaSuccess ||
      dalloc(&md->w16, md->P) != cudaSuccess || dalloc(&md->lpart, 2 * (size_t)md->max_blocks) != cudaSuccess ||
      dalloc(&md->loss, 1) != cudaSuccess)
    return bail(gfail(PDLP_ERR_OOM, "model allocation failed"));
  const size_t part_floats = std::max<size_t>((size_t)sm_count() * 2 * kDensePart,
                                              (size_t)2 * md->max_blocks * 65);
  if (dalloc(&md->part, std::max<size_t>(part_floats, (size_t)sm_count() * 2 * 7 * H)) != cudaSuccess)
    return bail(gfail(PDLP_ERR_OOM, "model allocation failed"));
  e = cudaFuncSetAttribute(k_gnn_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gnn_dense_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kBwdSmem);
  if (e != cudaSuccess) return bail(gfail(PDLP_ERR_CUDA, cudaGetErrorString(e)));
  // Xavier-uniform from SplitMix64, block by block in parameter order
  std::vector<float> th(md->P, 0.f);
  SplitMix64 r{seed};
  auto fill = [&](int off, int rows, int cols, int fan_in, int fan_out) {
    const double lim = std::sqrt(6.0 / (double)(fan_in + fan_out));
    for (int i = 0; i < rows * cols; ++i) th[off + i] = (float)((2.0 * r.uniform() - 1.0) * lim);
  };
  fill(kOff.W_vin, GNN_VAR_FEATURES, H, GNN_VAR_FEATURES, H);
  fill(kOff.W_cin, GNN_CON_FEATURES, H, GNN_CON_FEATURES, H);
  for (int k = 0; k < GNN_LAYERS; ++k) {
    fill(kOff.W_cc[k], H, H, H, H);
    fill(kOff.W_cv[k], H, H, H, H);
    fill(kOff.W_vv[k], H, H, H, H);
    fill(kOff.W_vc[k], H, H, H, H);
  }
  fill(kOff.w_x, 1, H, H, 1);
  fill(kOff.w_y, 1, H, H, 1);
  int rc = gnn_set_params(md, th.data());
  if (rc != PDLP_OK) return bail(rc);
  e = cudaMemsetAsync(md->grad, 0, sizeof(float) * md->P, md->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(md->m1, 0, sizeof(float) * md->P, md->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(md->m2, 0, sizeof(float) * md->P, md->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(md->s);
  if (e != cudaSuccess) return bail(gfail(PDLP_ERR_CUDA, cudaGetErrorString(e)));
  *out = md;
  return PDLP_OK;
}

int gnn_free(gnn_model* md) {
  if (!md) return PDLP_OK;
  if (md->s) cudaStreamSynchronize(md->s);
  free_scratch(md);
  void* ps[] = {md->theta, md->grad, md->m1, md->m2, md->w16, md->part, md->lpart, md->loss};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (md->s) cudaStreamDestroy(md->s);
  delete md;
  return PDLP_OK;
}

int gnn_get_params(const gnn_model* md, float* out) {
  RTRY(check_model(md));
  if (!out) return gfail(PDLP_ERR_INVALID_INPUT, "NULL output");
  GTRY(cudaMemcpyAsync(out, md->theta, sizeof(float) * md->P, cudaMemcpyDeviceToHost, md->s));
  GTRY(cudaStreamSynchronize(md->s));
  return PDLP_OK;
}

int gnn_set_params(gnn_model* md, const float* in) {
  RTRY(check_model(md));
  if (!in) return gfail(PDLP_ERR_INVALID_INPUT, "NULL input");
  for (int i = 0; i < md->P; ++i)
    if (!std::isfinite(in[i])) return gfail(PDLP_ERR_INVALID_INPUT, "non-finite parameter");
  GTRY(cudaMemcpyAsync(md->theta, in, sizeof(float) * md->P, cudaMemcpyHostToDevice, md->s));
  k_gnn_to_bf16<<<grid_rows(md->P, NB, sm_count() * 4), NB, 0, md->s>>>(md->P, md->theta, md->w16);
  GTRY(cudaGetLastError());
  GTRY(cudaStreamSynchronize(md->s));
  return PDLP_OK;
}

int gnn_get_grad(const gnn_model* md, float* out) {
  RTRY(check_model(md));
  if (!out) return gfail(PDLP_ERR_INVALID_INPUT, "NULL output");
  GTRY(cudaMemcpyAsync(out, md->grad, sizeof(float) * md->P, cudaMemcpyDeviceToHost, md->s));
  GTRY(cudaStreamSynchronize(md->s));
  return PDLP_OK;
}

int gnn_set_grad(gnn_model* md, const float* in) {
  RTRY(check_model(md));
  if (!in) return gfail(PDLP_ERR_INVALID_INPUT, "NULL input");
  GTRY(cudaMemcpyAsync(md->grad, in, sizeof(float) * md->P, cudaMemcpyHostToDevice, md->s));
  GTRY(cudaStreamSynchronize(md->s));
  return PDLP_OK;
}

int gnn_zero_grad(gnn_model* md) {
  RTRY(check_model(md));
  GTRY(cudaMemsetAsync(md->grad, 0, sizeof(float) * md->P, md->s));
  return PDLP_OK;
}

int gnn_save(const gnn_model* md, const char* path) {
  RTRY(check_model(md));
  if (!path) return gfail(PDLP_ERR_INVALID_INPUT, "NULL path");
  std::vector<float> buf(3 * (size_t)md->P);
  GTRY(cudaMemcpyAsync(buf.data(), md->theta, sizeof(float) * md->P, cudaMemcpyDeviceToHost, md->s));
  GTRY(cudaMemcpyAsync(buf.data() + md->P, md->m1, sizeof(float) * md->P, cudaMemcpyDeviceToHost, md->s));
  GTRY(cudaMemcpyAsync(buf.data() + 2 * (size_t)md->P, md->m2, sizeof(float) * md->P,
                       cudaMemcpyDeviceToHost, md->s));
  GTRY(cudaStreamSynchronize(md->s));
  FILE* f = fopen(path, "wb");
  if (!f) return gfail(PDLP_ERR_INVALID_INPUT, std::string("cannot open ") + path);
  const int64_t hdr[2] = {md->P, md->step};
  bool ok = fwrite("PDLPGNN1", 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? PDLP_OK : gfail(PDLP_ERR_INVALID_INPUT, std::string("write failed: ") + path);
}

int gnn_load(const char* path, gnn_model** out) {
  if (!path || !out) return gfail(PDLP_ERR_INVALID_INPUT, "NULL argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return gfail(PDLP_ERR_INVALID_INPUT, std::string("cannot open ") + path);
  char magic[8];
  int64_t hdr[2];
  std::vector<float> buf(3 * (size_t)kOff.total);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "PDLPGNN1", 8) == 0 &&
            fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == kOff.total &&
            fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) return gfail(PDLP_ERR_INVALID_INPUT, std::string("not a model file of this network: ") + path);
  gnn_model* md = nullptr;
  RTRY(gnn_create(0, &md));
  int rc = gnn_set_params(md, buf.data());
  if (rc == PDLP_OK) {
    cudaError_t e = cudaMemcpyAsync(md->m1, buf.data() + md->P, sizeof(float) * md->P,
                                    cudaMemcpyHostToDevice, md->s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(md->m2, buf.data() + 2 * (size_t)md->P, sizeof(float) * md->P,
                          cudaMemcpyHostToDevice, md->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(md->s);
    if (e != cudaSuccess) rc = gfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc != PDLP_OK) {
    gnn_free(md);
    return rc;
  }
  md->step = hdr[1];
  *out = md;
  return PDLP_OK;
}

int gnn_graph_create(gnn_model* md, const pdlp_csr* A, const double* b, const char* sense,
                     const double* c, const double* l, const double* u, gnn_graph** out) {
  RTRY(check_model(md));
  if (!out) return gfail(PDLP_ERR_INVALID_INPUT, "NULL output handle");
  *out = nullptr;
  gnn_graph* g = new gnn_graph();
  g->owner = md;
  cudaStream_t s = md->s;
  // the graph's own arrays and the feature pass's scratch share the LP's allocation
  const size_t M = A ? (size_t)std::max(A->m, 0) : 0, N = A ? (size_t)std::max(A->n, 0) : 0;
  Carve cv;
  const size_t o_idr = cv.take(4 * M), o_idc = cv.take(4 * N);
  const size_t o_fv = cv.take(4 * N * GNN_VAR_FEATURES), o_fc = cv.take(4 * M * GNN_CON_FEATURES);
  const size_t o_nr = cv.take(8 * M), o_nc = cv.take(8 * N), o_mx = cv.take(6 * 8);
  int rc = build_lp_dev(A, b, sense, c, l, u, s, &g->d, cv.off);
  if (rc != PDLP_OK) {
    gnn_graph_free(g);
    return rc;
  }
  const int m = g->d.m, n = g->d.n;
  unsigned char* ex = g->d.extra;
  g->inv_deg_r = (float*)(ex + o_idr);
  g->inv_deg_c = (float*)(ex + o_idc);
  g->fv = (float*)(ex + o_fv);
  g->fc = (float*)(ex + o_fc);
  double* nr = (double*)(ex + o_nr);
  double* nc = (double*)(ex + o_nc);
  unsigned long long* mx = (unsigned long long*)(ex + o_mx);
  unsigned long long hmx[6] = {};
  cudaError_t e = cudaMemsetAsync(mx, 0, 6 * sizeof(unsigned long long), s);
  const int G = sm_count() * 8;
  if (e == cudaSuccess && m > 0) {
    k_gnn_stats<<<grid_rows(m, NB, G), NB, 0, s>>>(m, g->d.a_ptr, g->d.a_val, g->d.b, nr,
                                                   g->inv_deg_r, mx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n > 0) {
    k_gnn_stats<<<grid_rows(n, NB, G), NB, 0, s>>>(n, g->d.t_ptr, g->d.t_val, g->d.c, nc,
                                                   g->inv_deg_c, mx + 3);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n > 0) {
    k_gnn_feat_v<<<grid_rows(n, NB, G), NB, 0, s>>>(n, g->d.t_ptr, g->d.c, g->d.l, g->d.u, nc, mx, g->fv);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && m > 0) {
    k_gnn_feat_c<<<grid_rows(m, NB, G), NB, 0, s>>>(m, g->d.a_ptr, g->d.b, g->d.kind, nr, mx, g->fc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    gnn_graph_free(g);
    return gfail(e == cudaErrorMemoryAllocation ? PDLP_ERR_OOM : PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  double cm;
  memcpy(&cm, &hmx[3], sizeof(double));
  g->cmax = std::max(cm, 1e-12);
  *out = g;
  return PDLP_OK;
}

int gnn_graph_set_labels(gnn_graph* g, const double* x_star, const double* y_star) {
  if (!g || !x_star || (!y_star && g->d.m > 0)) return gfail(PDLP_ERR_INVALID_INPUT, "NULL argument");
  RTRY(check_model(g->owner));
  const int n = g->d.n, m = g->d.m;
  std::vector<float> xs(std::max(n, 1)), ys(std::max(m, 1));
  std::vector<char> sense(std::max(m, 1));
  cudaStream_t s = g->owner->s;
  if (m > 0) {
    GTRY(cudaMemcpyAsync(sense.data(), g->d.sense, m, cudaMemcpyDeviceToHost, s));
    GTRY(cudaStreamSynchronize(s));
  }
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(x_star[j])) return gfail(PDLP_ERR_INVALID_INPUT, "non-finite x label");
    xs[j] = (float)x_star[j];
  }
  for (int i = 0; i < m; ++i) {
    if (!std::isfinite(y_star[i])) return gfail(PDLP_ERR_INVALID_INPUT, "non-finite y label");
    ys[i] = (float)((sense[i] == 'L' ? -y_star[i] : y_star[i]) / g->cmax);
  }
  if (!g->x_star) GTRY(dalloc(&g->x_star, n));
  if (!g->y_star) GTRY(dalloc(&g->y_star, m));
  GTRY(cudaMemcpyAsync(g->x_star, xs.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
  GTRY(cudaMemcpyAsync(g->y_star, ys.data(), sizeof(float) * m, cudaMemcpyHostToDevice, s));
  GTRY(cudaStreamSynchronize(s));
  g->has_labels = 1;
  return PDLP_OK;
}

int gnn_graph_features(const gnn_graph* g, float* fv, float* fc) {
  if (!g) return gfail(PDLP_ERR_INVALID_INPUT, "NULL graph");
  RTRY(check_model(g->owner));
  cudaStream_t s = g->owner->s;
  if (fv && g->d.n > 0)
    GTRY(cudaMemcpyAsync(fv, g->fv, sizeof(float) * g->d.n * GNN_VAR_FEATURES, cudaMemcpyDeviceToHost, s));
  if (fc && g->d.m > 0)
    GTRY(cudaMemcpyAsync(fc, g->fc, sizeof(float) * g->d.m * GNN_CON_FEATURES, cudaMemcpyDeviceToHost, s));
  GTRY(cudaStreamSynchronize(s));
  return PDLP_OK;
}

int gnn_graph_free(gnn_graph* g) {
  if (!g) return PDLP_OK;
  // cudaFree waits for the device; the owner is not touched (it may be gone).  The degree
  // and feature arrays live in the LP's allocation; the labels have their own.
  g->d.release();
  void* ps[] = {g->x_star, g->y_star};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete g;
  return PDLP_OK;
}

int gnn_forward(gnn_model* md, gnn_graph* g, double* x_out, double* y_out, double* loss) {
  RTRY(check_model(md));
  if (!g || g->owner != md) return gfail(PDLP_ERR_INVALID_INPUT, "graph does not belong to this model");
  const bool lab = g->has_labels != 0;
  RTRY(forward(md, g, true, lab, false));
  cudaStream_t s = md->s;
  if (x_out && g->d.n > 0)
    GTRY(cudaMemcpyAsync(x_out, md->xpred, sizeof(double) * g->d.n, cudaMemcpyDeviceToHost, s));
  if (y_out && g->d.m > 0)
    GTRY(cudaMemcpyAsync(y_out, md->ypred, sizeof(double) * g->d.m, cudaMemcpyDeviceToHost, s));
  double hl = NAN;
  if (lab) GTRY(cudaMemcpyAsync(&hl, md->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
  GTRY(cudaStreamSynchronize(s));
  if (loss) *loss = hl;
  return PDLP_OK;
}

int gnn_backward(gnn_model* md, gnn_graph* g, double scale, double* loss) {
  RTRY(check_model(md));
  if (!g || g->owner != md) return gfail(PDLP_ERR_INVALID_INPUT, "graph does not belong to this model");
  if (!g->has_labels) return gfail(PDLP_ERR_INVALID_INPUT, "graph has no labels");
  RTRY(backward(md, g, (float)scale));
  double hl = NAN;
  GTRY(cudaMemcpyAsync(&hl, md->loss, sizeof(double), cudaMemcpyDeviceToHost, md->s));
  GTRY(cudaStreamSynchronize(md->s));
  if (loss) *loss = hl;
  return PDLP_OK;
}

int gnn_default_adam(gnn_adam* a) {
  if (!a) return gfail(PDLP_ERR_INVALID_INPUT, "NULL argument");
  a->struct_size = sizeof(gnn_adam);
  a->lr = 1e-3;
  a->beta1 = 0.9;
  a->beta2 = 0.999;
  a->eps = 1e-8;
  return PDLP_OK;
}

int gnn_adam_step(gnn_model* md, const gnn_adam* a) {
  RTRY(check_model(md));
  if (!a || a->struct_size != sizeof(gnn_adam)) return gfail(PDLP_ERR_INVALID_INPUT, "bad gnn_adam");
  if (!(a->lr > 0) || !(a->beta1 >= 0 && a->beta1 < 1) || !(a->beta2 >= 0 && a->beta2 < 1) ||
      !(a->eps >= 0))
    return gfail(PDLP_ERR_INVALID_INPUT, "Adam settings out of range");
  RTRY(adam_step(md, a));
  GTRY(cudaStreamSynchronize(md->s));
  return PDLP_OK;
}

int gnn_default_train(gnn_train_params* t) {
  if (!t) return gfail(PDLP_ERR_INVALID_INPUT, "NULL argument");
  t->struct_size = sizeof(gnn_train_params);
  t->epochs = 30;
  t->batch = 4;
  gnn_default_adam(&t->adam);
  t->lr_decay = 0.95;
  t->seed = 1;
  return PDLP_OK;
}

int gnn_train(gnn_model* md, gnn_graph* const* graphs, int count, const gnn_train_params* t,
              double* epoch_loss) {
  RTRY(check_model(md));
  if (!graphs || count <= 0 || !t || t->struct_size != sizeof(gnn_train_params) || t->epochs < 0 ||
      t->batch <= 0 || t->adam.struct_size != sizeof(gnn_adam))
    return gfail(PDLP_ERR_INVALID_INPUT, "bad training arguments");
  for (int i = 0; i < count; ++i)
    if (!graphs[i] || graphs[i]->owner != md || !graphs[i]->has_labels)
      return gfail(PDLP_ERR_INVALID_INPUT, "graph " + std::to_string(i) + " is missing, foreign or unlabelled");
  double* hist = nullptr;
  GTRY(dalloc(&hist, count));
  std::vector<double> h(count);
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  SplitMix64 r{t->seed};
  gnn_adam a = t->adam;
  int rc = PDLP_OK;
  for (int ep = 0; ep < t->epochs && rc == PDLP_OK; ++ep) {
    for (int i = count - 1; i > 0; --i) {
      const int j = (int)(r.uniform() * (double)(i + 1));
      std::swap(order[i], order[j]);
    }
    for (int b0 = 0; b0 < count && rc == PDLP_OK; b0 += t->batch) {
      const int b1 = std::min(count, b0 + t->batch);
      if (cudaMemsetAsync(md->grad, 0, sizeof(float) * md->P, md->s) != cudaSuccess) {
        rc = gfail(PDLP_ERR_CUDA, "memset");
        break;
      }
      for (int k = b0; k < b1 && rc == PDLP_OK; ++k) {
        rc = backward(md, graphs[order[k]], 1.0f / (float)(b1 - b0));
        if (rc == PDLP_OK &&
            cudaMemcpyAsync(hist + k, md->loss, sizeof(double), cudaMemcpyDeviceToDevice, md->s) != cudaSuccess)
          rc = gfail(PDLP_ERR_CUDA, "loss copy");
      }
      if (rc == PDLP_OK) rc = adam_step(md, &a);
    }
    if (rc == PDLP_OK) {
      if (cudaMemcpyAsync(h.data(), hist, sizeof(double) * count, cudaMemcpyDeviceToHost, md->s) != cudaSuccess ||
          cudaStreamSynchronize(md->s) != cudaSuccess)
        rc = gfail(PDLP_ERR_CUDA, "loss read-back");
      else if (epoch_loss) {
        double s = 0.0;
        for (double v : h) s += v;
        epoch_loss[ep] = s / count;
      }
    }
    a.lr *= t->lr_decay;
  }
  cudaStreamSynchronize(md->s);
  cudaFree(hist);
  return rc;
}

int pdlp_start_kkt(const pdlp_csr* A, const double* b, const char* sense, const double* c,
                   const double* l, const double* u, const double* x0, const double* y0,
                   double* kkt_out) {
  if (!kkt_out || !x0 || (!y0 && A && A->m > 0)) return gfail(PDLP_ERR_INVALID_INPUT, "NULL argument");
  cudaStream_t s = nullptr;
  GTRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  LpDev d;
  double *x = nullptr, *y = nullptr, *part = nullptr, *out = nullptr;
  int rc = build_lp_dev(A, b, sense, c, l, u, s, &d);
  cudaError_t e = cudaSuccess;
  if (rc == PDLP_OK) {
    e = dalloc(&x, d.n);
    if (e == cudaSuccess) e = dalloc(&y, d.m);
    if (e == cudaSuccess) e = dalloc(&part, start_kkt_part_doubles());
    if (e == cudaSuccess) e = dalloc(&out, 4);
    if (e == cudaSuccess && d.n > 0)
      e = cudaMemcpyAsync(x, x0, sizeof(double) * d.n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && d.m > 0)
      e = cudaMemcpyAsync(y, y0, sizeof(double) * d.m, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = gfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc == PDLP_OK) rc = start_kkt(d, x, y, 0, part, out, s);
  if (rc == PDLP_OK) {
    e = cudaMemcpyAsync(kkt_out, out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = gfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaStreamSynchronize(s);
  for (void* p : {(void*)x, (void*)y, (void*)part, (void*)out})
    if (p) cudaFree(p);
  d.release();
  cudaStreamDestroy(s);
  return rc;
}

int pdlp_solve_warm(gnn_model* md, const pdlp_csr* A, const double* b, const char* sense,
                    const double* c, const double* l, const double* u, const pdlp_params* p,
                    double* x_out, double* y_out, pdlp_result* r, gnn_warm_info* info) {
  if (!md)
    return pdlp_solve(A, b, sense, c, l, u, p, nullptr, nullptr, x_out, y_out, r, nullptr);
  RTRY(check_model(md));
  if (!r || !x_out || (!y_out && A && A->m > 0)) return gfail(PDLP_ERR_INVALID_INPUT, "NULL output");
  const auto t0 = std::chrono::steady_clock::now();
  gnn_graph* g = nullptr;
  RTRY(gnn_graph_create(md, A, b, sense, c, l, u, &g));
  cudaStream_t s = md->s;
  const int n = g->d.n, m = g->d.m;
  double *xc = nullptr, *yc = nullptr, *part = nullptr, *kk = nullptr, *xo = nullptr, *yo = nullptr;
  double* buf = nullptr;  // the six scratch vectors in one allocation
  double hk[8] = {};
  int rc = forward(md, g, true, false, false);
  cudaError_t e = cudaSuccess;
  if (rc == PDLP_OK) {
    Carve cv;
    const size_t o_xc = cv.take(8 * (size_t)n), o_yc = cv.take(8 * (size_t)m);
    const size_t o_part = cv.take(8 * start_kkt_part_doubles()), o_kk = cv.take(8 * 8);
    const size_t o_xo = cv.take(8 * (size_t)n), o_yo = cv.take(8 * (size_t)m);
    e = cudaMalloc((void**)&buf, cv.off);
    if (e == cudaSuccess) {
      unsigned char* p0 = (unsigned char*)buf;
      xc = (double*)(p0 + o_xc);
      yc = (double*)(p0 + o_yc);
      part = (double*)(p0 + o_part);
      kk = (double*)(p0 + o_kk);
      xo = (double*)(p0 + o_xo);
      yo = (double*)(p0 + o_yo);
    } else {
      rc = gfail(PDLP_ERR_OOM, cudaGetErrorString(e));
    }
  }
  if (rc == PDLP_OK) rc = start_kkt(g->d, md->xpred, md->ypred, 0, part, kk, s);
  if (rc == PDLP_OK) rc = start_kkt(g->d, xc, yc, 1, part, kk + 4, s);
  if (rc == PDLP_OK) {
    e = cudaMemcpyAsync(hk, kk, sizeof(hk), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = gfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  const double predict_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const bool warm = rc == PDLP_OK && hk[3] < hk[7];
  if (rc == PDLP_OK) {
    // the start point is the one chosen above; the primal weight always comes from the
    // projected prediction's norms (pdlp_solve_hinted)
    pdlp_csr Ad{m, n, (int64_t)g->d.nnz, g->d.ptr64, g->d.a_col, g->d.a_val};
    rc = pdlp::solve_device_hint(&Ad, g->d.b, g->d.sense, g->d.c, g->d.l, g->d.u, p,
                                 warm ? md->xpred : nullptr, warm ? md->ypred : nullptr,
                                 md->xpred, md->ypred, xo, yo, r, s);
  }
  if (rc == PDLP_OK) {
    if (n > 0) e = cudaMemcpyAsync(x_out, xo, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && m > 0 && y_out)
      e = cudaMemcpyAsync(y_out, yo, sizeof(double) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = gfail(PDLP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (info) {
    info->used_warm = warm ? 1 : 0;
    info->warm_rel_kkt = hk[3];
    info->cold_rel_kkt = hk[7];
    info->predict_s = predict_s;
  }
  cudaStreamSynchronize(s);
  if (buf) cudaFree(buf);
  gnn_graph_free(g);
  return rc;
}

}  // extern "C"
