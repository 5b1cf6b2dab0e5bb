// Warp-tile step kernels for float32 iterates (rows A4-A7 of the hot path).
//
// The same attempt as k_primal / k_dual (iter_kernels.cuh) and k_tile
// (tile_kernels.cuh), with the work cut into warp-sized items at setup
// (setup_tiles with the warp shape): a tile is at most 32 consecutive rows whose
// nonzeros start inside one window of W entries (64 <= W <= 256, so fewer than
// W + 256 nonzeros), a row longer than 256 entries is cut into slices of at most
// W entries.  Every warp of the grid owns the items w, w + T, w + 2T, ... (T warps
// in all) and works on its own, with no block-wide synchronisation:
//   1. the item's descriptor (prefetched one item ahead), then, all issued
//      together, the rows' constant and iterate entries (one row per lane), the
//      row pointers, and the item's column indices and values in passes of
//      8 per lane;
//   2. the gathers at those indices (8 per lane in flight), the products into the
//      warp's shared-memory buffer;
//   3. one lane per row sums its products in storage order and updates the row;
//      outputs are coalesced stores.
// Many independent warps per SM, each with its whole item's streams in flight,
// keep the memory system busy without a deep staging ring.  A slice's products are
// summed by its warp; the row is finished by the warp that completes its last slice
// (an atomic ticket; the slices' partials added in slice order).  Step-rule partial
// sums are kept per warp and written once per (warp, LP) run into the slot of the
// run's first item; long rows write theirs into a slot of their own; k_decide adds
// them in index order.  Constant data of a warp's first item is loaded before the
// dependent-launch wait.
#pragma once

#include "tile_kernels.cuh"

namespace pdlp {

constexpr int kWarpTileNnz = kWarpTileWindowMax + kLongRow;  // nonzeros of an item, at most
constexpr int kWarpPass = 8;                                 // entries per lane per pass

template <typename V>
__device__ __forceinline__ float ldv(const V* v, int p) {
  return ldv_f<V>(v, p);
}

template <typename V, bool IMPLICIT, bool DUAL>
__global__ void __launch_bounds__(kBlock, 4) k_wtile(IterData<float, V> d) {
  __shared__ float prod_a[kWarps][kWarpTileNnz];
  __shared__ float prod_b[DUAL ? kWarps : 1][DUAL ? kWarpTileNnz : 1];
  const TileSet& ts = DUAL ? d.ta : d.tt;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int T = gridDim.x * kWarps;
  const int w0 = blockIdx.x * kWarps + warp;
  const int* ptr = DUAL ? d.a_ptr : d.t_ptr;
  const int* col = DUAL ? d.a_col : d.t_col;
  const V* val = DUAL ? d.a_val : d.t_val;
  float* pa = prod_a[warp];
  float* pb = prod_b[DUAL ? warp : 0];

  // constant row entries of an item's rows, one row per lane (primal: c, l, u, tw;
  // dual: q, sw and the row kind), and its row pointers
  struct RowConst {
    float c0, c1, c2, c3;
    int kind, p0, p1;
  };
  auto row_const = [&](const TileItem& it) -> RowConst {
    RowConst rc{0.f, 0.f, 0.f, 1.f, 0, 0, 0};
    const int r = it.r0 + lane;
    if (it.first < 0 && r < it.r1) {
      if (DUAL) {
        rc.c0 = __ldg(d.q + r);
        if (IMPLICIT) rc.c3 = __ldg(d.sw + r);
        rc.kind = __ldg(d.row_kind + r);
      } else {
        rc.c0 = __ldg(d.c + r);
        rc.c1 = __ldg(d.l + r);
        rc.c2 = __ldg(d.u + r);
        if (IMPLICIT) rc.c3 = __ldg(d.tw + r);
      }
      rc.p0 = __ldg(ptr + r);
      rc.p1 = __ldg(ptr + r + 1);
    }
    return rc;
  };

  TileItem it{};
  RowConst rc{};
  if (w0 < ts.n) {
    it = ts.item[w0];
    rc = row_const(it);
  }
  pdl_enter();
  if (w0 >= ts.n) return;

  float acc1 = 0.0f, acc2 = 0.0f;  // this lane's share of the current (warp, LP) run
  int run_lp = -1, run_slot = -1, run_go = 0;
  StageMeta mt{};
  int mt_lp = -1;
  auto flush = [&]() {
    if (run_lp >= 0 && run_go) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
        acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
      }
      if (lane == 0) ts.part[run_slot] = make_float2(acc1, acc2);
    }
    acc1 = acc2 = 0.0f;
  };

  for (int i = w0; i < ts.n; i += T) {
    const bool has_next = i + T < ts.n;
    const TileItem nx = has_next ? ts.item[i + T] : TileItem{};
    if (it.lp != mt_lp) {
      mt = item_meta<V, DUAL>(d, it.lp);
      mt_lp = it.lp;
    }
    if (it.lp != run_lp) {
      flush();
      run_lp = it.lp;
      run_slot = i;
      run_go = mt.go;
    }
    if (mt.go) {
      // iterate entries of the lane's row (issued with the streams below)
      const int r = it.r0 + lane;
      const bool row = it.first < 0 && r < it.r1;
      float xo = 0.0f, so = 0.0f;
      if (row) {
        if (DUAL) {
          xo = (mt.cur ? d.y[1] : d.y[0])[r];
          if (mt.pw != 0.0f) so = d.sum_y[r];
        } else {
          xo = (mt.cur ? d.x[1] : d.x[0])[r].x;
          if (mt.pw != 0.0f) so = d.sum_x[r];
        }
      }
      // products of the item's nonzeros, kWarpPass per lane per pass
      const float2* xg = mt.cur ? d.x[0] : d.x[1];  // dual: x' of this attempt
      const float* yg = mt.cur ? d.y[1] : d.y[0];    // primal: current y
      const int nz = it.ne - it.nb;
      for (int q = lane; q < nz; q += 32 * kWarpPass) {
        int cj[kWarpPass];
        float vv[kWarpPass];
#pragma unroll
        for (int k = 0; k < kWarpPass; ++k) {
          const int e = q + 32 * k;
          cj[k] = e < nz ? __ldg(col + it.nb + e) : 0;
          vv[k] = e < nz ? ldv<V>(val, it.nb + e) : 0.0f;
        }
        if (DUAL) {
          float2 g[kWarpPass];
#pragma unroll
          for (int k = 0; k < kWarpPass; ++k) g[k] = q + 32 * k < nz ? xg[cj[k]] : make_float2(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < kWarpPass; ++k) {
            const int e = q + 32 * k;
            if (e < nz) {
              pa[e] = vv[k] * g[k].x;
              pb[e] = vv[k] * g[k].y;
            }
          }
        } else {
          float g[kWarpPass];
#pragma unroll
          for (int k = 0; k < kWarpPass; ++k) g[k] = q + 32 * k < nz ? yg[cj[k]] : 0.0f;
#pragma unroll
          for (int k = 0; k < kWarpPass; ++k) {
            const int e = q + 32 * k;
            if (e < nz) pa[e] = vv[k] * g[k];
          }
        }
      }
      __syncwarp();
      if (it.first < 0) {
        if (row) {
          float a = 0.0f, b = 0.0f;
          for (int p = rc.p0 - it.nb; p < rc.p1 - it.nb; ++p) {
            a += pa[p];
            if (DUAL) b += pb[p];
          }
          if (DUAL) {
            const float2 tm = dual_row<IMPLICIT>(a, b, rc.c0, rc.c3, rc.kind, xo, so, mt.step,
                                                 mt.pw, mt.cur ? d.y[0] : d.y[1], d.sum_y, r);
            acc1 += tm.x;
            acc2 += tm.y;
          } else {
            acc1 += primal_row<IMPLICIT>(a, rc.c0, rc.c1, rc.c2, rc.c3, xo, so, mt.step, mt.pw,
                                         mt.cur ? d.x[0] : d.x[1], d.sum_x, r);
          }
        }
      } else {
        // slice of a long row: the warp's sum, then the ticket
        float a = 0.0f, b = 0.0f;
        for (int p = lane; p < nz; p += 32) {
          a += pa[p];
          if (DUAL) b += pb[p];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        int last = 0;
        if (lane == 0) {
          ts.rowpart[i] = make_float2(a, b);
          __threadfence();
          last = atomicAdd(&ts.ticket[it.first], 1) == it.nsl - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {  // the last slice: the warp adds the slices' partials, lane 0 finishes
          __threadfence();
          float ra = 0.0f, rb = 0.0f;
          for (int k = lane; k < it.nsl; k += 32) {
            const float2 pv = __ldcg(ts.rowpart + it.first + k);
            ra += pv.x;
            rb += pv.y;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            ra += __shfl_xor_sync(0xffffffffu, ra, o);
            rb += __shfl_xor_sync(0xffffffffu, rb, o);
          }
          if (lane == 0) {
            const int rr = it.r0;
            if (DUAL) {
              const float* y = mt.cur ? d.y[1] : d.y[0];
              ts.lterm[it.lid] = dual_row<IMPLICIT>(
                  ra, rb, d.q[rr], IMPLICIT ? d.sw[rr] : 1.0f, d.row_kind[rr], y[rr],
                  mt.pw != 0.0f ? d.sum_y[rr] : 0.0f, mt.step, mt.pw, mt.cur ? d.y[0] : d.y[1],
                  d.sum_y, rr);
            } else {
              const float2* x = mt.cur ? d.x[1] : d.x[0];
              const float tm = primal_row<IMPLICIT>(
                  ra, d.c[rr], d.l[rr], d.u[rr], IMPLICIT ? d.tw[rr] : 1.0f, x[rr].x,
                  mt.pw != 0.0f ? d.sum_x[rr] : 0.0f, mt.step, mt.pw, mt.cur ? d.x[0] : d.x[1],
                  d.sum_x, rr);
              ts.lterm[it.lid] = make_float2(tm, 0.0f);
            }
            ts.ticket[it.first] = 0;  // ready for the next launch
          }
        }
      }
      __syncwarp();  // the buffer is rewritten by the next item
    }
    if (has_next) {
      it = nx;
      rc = row_const(it);
    }
  }
  flush();
}

}  // namespace pdlp
