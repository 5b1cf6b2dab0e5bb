// Staged tile step kernels for float32 iterates (rows A4-A7 of the hot path).
//
// The same attempt as k_primal / k_dual (iter_kernels.cuh) -- the projected
// primal step x' = proj_[l,u](x - tau (c - K^T y)) over the rows of A^T, the
// extrapolated dual step y' = proj_Y(y + sigma (q - K x' - K dx)) over the rows
// of A, the partial sums of the adaptive step rule -- organised around the
// Tensor Memory Accelerator's bulk copies instead of per-thread index chains.
//
// Work items.  The rows of a matrix are cut into items at setup
// (setup_tiles): a TILE is a run of at most kTileRows consecutive short rows
// whose nonzeros start inside one window of W entries (so a tile holds fewer
// than W + kLongRow nonzeros); a row longer than kLongRow is cut into SLICES of
// at most W entries, one item each.  Items never straddle two LPs of a batch.
//
// Staging.  A block owns the items b, b + G, b + 2G, ... of the grid's G
// blocks, in that order, and streams each one through a ring of kStages shared
// memory stages with 1-D bulk copies (cp.async.bulk, completion counted on an
// mbarrier): the item's row pointers, column indices and values and its rows'
// constant vectors (c, l, u, step weights / q, step weights, row kinds) on one
// barrier, the rows' iterate entries (x pairs, running sums / y, running sums)
// on a second.  Constant data does not change during the iteration phase, so
// the first stages are requested BEFORE the dependent-launch wait and arrive
// while the preceding kernel drains; iterate data is requested after it.
//
// Per item, with the stage in shared memory:
//   phase 1  one thread per nonzero (kMaxPerThread per thread, all issued before
//            any is used): gather the vector entry at the staged column index and
//            write the product with the staged value back into the stage;
//   phase 2  one thread per row: the row's products summed in storage order,
//            then the row's update from the staged vectors; outputs are
//            coalesced stores.
// A slice's products are summed by the block; the row is finished by whichever
// block completes its last slice (an atomic ticket per row; the finisher sums
// the slices' partials in slice order), so every row sum has one fixed order.
// Partial sums of the step rule are kept per thread across a block's items of
// one LP and reduced once per (block, LP) run into the slot of the run's first
// item; long rows write theirs into a slot of their own.  k_decide sums the
// slots of each LP in index order: the result does not depend on timing.
//
// Every wait on an mbarrier is bounded: a block that gives up records
// kStatusWaitFailed in its LP's state, waits (bounded again) for the copies it
// issued, and returns.
#pragma once

#include <type_traits>

#include "iter_kernels.cuh"

namespace pdlp {

constexpr int kTileNnz = kTileWindowMax + kLongRow;  // nonzeros of an item, at most
constexpr int kMaxPerThread = (kTileNnz + kBlock - 1) / kBlock;
constexpr int kNzSlots = kTileNnz + 16;   // staged nonzero slots (8-entry alignment each end)
constexpr int kRowSlots = kTileRows + 32;  // staged row slots (16-byte alignment each end)
constexpr int kPtrSlots = kTileRows + 8;   // staged row pointers (r1 - r0 + 1, 4-aligned)
constexpr long long kTileSpinLimit = 1LL << 22;  // polls of one mbarrier wait
constexpr int kTileStages = 2;                   // shared-memory stages per block
// a stage's facts are written after the barrier that ends its previous use and read
// one loop iteration later, after further barriers: two stages at least
static_assert(kTileStages >= 2, "the stage ring needs two stages");

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// true once the barrier's phase with the given parity has completed
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false if the limit ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (long long k = 0; k < kTileSpinLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 1-D bulk copy global -> shared, completion on `bar` (16-byte aligned, bytes % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) writes into the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Range [lo, hi) of an array of `esize`-byte elements widened to 16-byte
// boundaries: first element `a`, element count `cnt` (a multiple of 16 / esize).
// Workspace arrays start on 256-byte boundaries, so the widened end stays inside
// the array's own padding.
struct Span16 {
  int a, cnt;
};
__device__ __forceinline__ Span16 span16(int lo, int hi, int esize) {
  const int g = 16 / esize;
  const int a = lo & ~(g - 1);
  const int b = (hi + g - 1) & ~(g - 1);
  return Span16{a, b - a};
}

// ---------------------------------------------------------------- stages
// Shared-memory layout of one stage; every region 16-byte aligned.
template <typename V, bool DUAL>
struct StageLayout {
  static constexpr int kValBytes = std::is_same<V, Pattern>::value ? 0 : (int)sizeof(V);
  static constexpr int ptr = 0;                                  // int [kPtrSlots]
  static constexpr int col = ptr + kPtrSlots * 4;                // int [kNzSlots], products a
  static constexpr int val = col + kNzSlots * 4;                 // V [kNzSlots]
  static constexpr int prb = val + ((kNzSlots * kValBytes + 15) & ~15);  // float [kNzSlots] (dual)
  static constexpr int rows = prb + (DUAL ? kNzSlots * 4 : 0);
  // primal rows: c, l, u, tw, sum_x (float), x pairs (float2)
  // dual rows:   q, sw, y, sum_y (float), row kind (byte)
  static constexpr int r0 = rows;
  static constexpr int r1 = r0 + kRowSlots * 4;
  static constexpr int r2 = r1 + kRowSlots * 4;
  static constexpr int r3 = r2 + kRowSlots * 4;
  static constexpr int r4 = r3 + kRowSlots * 4;
  static constexpr int r5 = r4 + kRowSlots * 4;  // primal: x pairs; dual: row kinds
  static constexpr int bytes = r5 + (DUAL ? kRowSlots : kRowSlots * 8);
};

template <typename V>
__device__ __forceinline__ float stage_val(const unsigned char* s, int k);
template <>
__device__ __forceinline__ float stage_val<float>(const unsigned char* s, int k) {
  return reinterpret_cast<const float*>(s)[k];
}
template <>
__device__ __forceinline__ float stage_val<__nv_bfloat16>(const unsigned char* s, int k) {
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(s)[k]);
}
template <>
__device__ __forceinline__ float stage_val<Pattern>(const unsigned char*, int) {
  return 1.0f;
}

// Per-stage facts the producing thread records for the consumers.
struct StageMeta {
  int go;     // the item's LP steps in this attempt (else the item is skipped)
  int cur;    // which iterate buffers are current for the item's LP
  float step; // tau (primal) or sigma (dual) of the item's LP
  float pw;   // pending averaging weight of the item's LP (0: none)
};

// Requests the constant data of item `it` into stage `s` (one thread): row
// pointers, column indices, values, and the rows' constant vectors
// (primal c, l, u[, tw]; dual q[, sw] and the row kinds).
template <typename V, bool DUAL, bool IMPLICIT>
__device__ __forceinline__ void issue_const(unsigned char* s, const TileItem& it,
                                           const IterData<float, V>& d, unsigned long long* bar) {
  using L = StageLayout<V, DUAL>;
  const int* ptr = DUAL ? d.a_ptr : d.t_ptr;
  const int* col = DUAL ? d.a_col : d.t_col;
  const V* val = DUAL ? d.a_val : d.t_val;
  const Span16 sp = span16(it.r0, it.r1 + 1, 4);
  const int za = it.nb & ~7, zb = (it.ne + 7) & ~7;
  const Span16 sr = span16(it.r0, it.r1, 4);
  constexpr int ncr = DUAL ? (IMPLICIT ? 2 : 1) : (IMPLICIT ? 4 : 3);
  const float* cr[4] = {DUAL ? d.q : d.c, DUAL ? d.sw : d.l, d.u, d.tw};
  unsigned bytes = 4u * (unsigned)sp.cnt;
  if (zb > za) bytes += (unsigned)((4 + L::kValBytes) * (zb - za));
  bytes += 4u * (unsigned)(ncr * sr.cnt);
  Span16 sk{0, 0};
  if (DUAL) {
    sk = span16(it.r0, it.r1, 1);
    bytes += (unsigned)sk.cnt;
  }
  mbar_arrive_expect_tx(bar, bytes);
  bulk_g2s(s + L::ptr, ptr + sp.a, 4u * sp.cnt, bar);
  if (zb > za) {
    bulk_g2s(s + L::col, col + za, 4u * (zb - za), bar);
    if (L::kValBytes) bulk_g2s(s + L::val, val + za, (unsigned)(L::kValBytes * (zb - za)), bar);
  }
  if (sr.cnt) {
#pragma unroll
    for (int k = 0; k < ncr; ++k) bulk_g2s(s + L::r0 + k * (kRowSlots * 4), cr[k] + sr.a, 4u * sr.cnt, bar);
    if (DUAL) bulk_g2s(s + L::r5, d.row_kind + sk.a, (unsigned)sk.cnt, bar);
  }
}

// Requests the iterate data of item `it` into stage `s` (one thread): the rows'
// current entries (primal x pairs, dual y) and, with a pending weight, their
// running sums; an item whose LP does not step this attempt gets none.  Always
// the stage's second arrival of the use.
template <typename V, bool DUAL>
__device__ __forceinline__ void issue_iter(unsigned char* s, const TileItem& it,
                                           const IterData<float, V>& d, const StageMeta& mt,
                                           unsigned long long* bar) {
  using L = StageLayout<V, DUAL>;
  const Span16 s4 = span16(it.r0, it.r1, 4);
  const Span16 s8 = span16(it.r0, it.r1, 8);
  const bool with_sum = mt.pw != 0.0f;
  const unsigned bytes =
      mt.go ? (with_sum ? 4u * s4.cnt : 0u) + (DUAL ? 4u * s4.cnt : 8u * s8.cnt) : 0u;
  mbar_arrive_expect_tx(bar, bytes);
  if (bytes == 0) return;
  if (DUAL) {
    const float* y = mt.cur ? d.y[1] : d.y[0];
    bulk_g2s(s + L::r2, y + s4.a, 4u * s4.cnt, bar);
    if (with_sum) bulk_g2s(s + L::r4, d.sum_y + s4.a, 4u * s4.cnt, bar);
  } else {
    const float2* x = mt.cur ? d.x[1] : d.x[0];
    bulk_g2s(s + L::r5, x + s8.a, 8u * s8.cnt, bar);
    if (with_sum) bulk_g2s(s + L::r4, d.sum_x + s4.a, 4u * s4.cnt, bar);
  }
}

// The state of an item's LP as the step kernels see it after the dependent-launch wait.
template <typename V, bool DUAL>
__device__ __forceinline__ StageMeta item_meta(const IterData<float, V>& d, int lp) {
  const DevState* st = d.st + lp;
  StageMeta m;
  m.go = (st->status == 0 && !st->check_due) ? 1 : 0;
  m.cur = st->cur;
  m.step = DUAL ? st->sigma_f : st->tau_f;
  m.pw = st->pw_f;
  return m;
}

// The update of one row from its sums (the same arithmetic as k_primal / k_dual):
// primal: acc_a = (K^T y)_j; writes x'_j and the pair, returns the ||dx||^2 term.
// dual: acc_a = (K x')_i, acc_b = (K dx)_i; writes y'_i, returns (||dy||^2, dy K dx) terms.
template <bool IMPLICIT>
__device__ __forceinline__ float primal_row(float aty, float c, float l, float u, float tw, float xo,
                                            float sx, float tau, float pw, float2* xn, float* sum_x,
                                            int j) {
  const float g = c - aty;
  const float step = IMPLICIT ? tau * tw : tau;
  const float xv = clampv(xo - step * g, l, u);
  const float dd = xv - xo;
  xn[j] = make_float2(xv, dd);
  if (pw != 0.0f) sum_x[j] = sx + pw * xo;
  return IMPLICIT ? dd * dd / tw : dd * dd;
}

template <bool IMPLICIT>
__device__ __forceinline__ float2 dual_row(float kx, float kdx, float q, float sw, int kind,
                                           float yo, float sy, float sigma, float pw, float* yn,
                                           float* sum_y, int i) {
  const float kxbar = kx + kdx;
  const float step = IMPLICIT ? sigma * sw : sigma;
  float yv = yo + step * (q - kxbar);
  if (kind != 1) yv = fmaxf(yv, 0.0f);
  yn[i] = yv;
  if (pw != 0.0f) sum_y[i] = sy + pw * yo;
  const float dd = yv - yo;
  return make_float2(IMPLICIT ? dd * dd / sw : dd * dd, dd * kdx);
}

// ---------------------------------------------------------------- the kernel
// DUAL = false: the primal step over the items of A^T (gathers y);
// DUAL = true:  the dual step over the items of A (gathers the (x', dx) pairs).
//
// The block's warps consume a staged item independently: warp w owns the item's
// rows [r0 + 32 w, r0 + 32 w + 32) -- their nonzeros are one contiguous run of the
// stage -- gathers for them, sums them and updates them; only __syncwarp orders a
// warp's own phases.  A warp then releases the stage (a shared-memory count) and the
// warp that releases it last requests the stage's next item, so no warp waits for
// another except through the data it needs.  A slice is shared by the 8 warps
// (one part of its nonzeros each); the last warp to finish its part adds the 8
// partial sums in warp order.  Step-rule partial sums are kept per warp and written
// once per (block, LP) run to the warp's slot of the run's first item.
template <typename V, bool IMPLICIT, bool DUAL>
__global__ void __launch_bounds__(kBlock, 4) k_tile(IterData<float, V> d) {
  using L = StageLayout<V, DUAL>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned long long bar_full[kTileStages];
  __shared__ StageMeta meta[kTileStages];
  __shared__ int released[kTileStages];   // warps done with the stage's current item
  __shared__ int slice_done[kTileStages];  // warps done with a slice's partial sum
  __shared__ float2 slice_part[kTileStages][kWarps];
  __shared__ int issued[kTileStages];      // uses of the stage requested so far
  __shared__ int fail;
  const TileSet& ts = DUAL ? d.ta : d.tt;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int nmine = b < ts.n ? (ts.n - 1 - b) / G + 1 : 0;
  if (nmine == 0) return;
  const int npre = nmine < kTileStages ? nmine : kTileStages;
  if (tid == 0) {
    for (int s = 0; s < kTileStages; ++s) {
      mbar_init(&bar_full[s], 2);  // two arrivals per use: constant data, iterate data
      released[s] = 0;
      slice_done[s] = 0;
      issued[s] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async_smem();
    fail = 0;
  }
  __syncthreads();
  // constant data of the first stages: independent of the preceding kernels
  if (tid == 0)
    for (int s = 0; s < npre; ++s) {
      issue_const<V, DUAL, IMPLICIT>(smem + s * L::bytes, ts.item[b + s * G], d, &bar_full[s]);
      issued[s] = 1;
    }
  pdl_enter();
  if (tid == 0)
    for (int s = 0; s < npre; ++s) {
      const TileItem it = ts.item[b + s * G];
      meta[s] = item_meta<V, DUAL>(d, it.lp);
      issue_iter<V, DUAL>(smem + s * L::bytes, it, d, meta[s], &bar_full[s]);
    }
  // (the meta writes are published by the arrivals; consumers read them after the wait)

  float acc1 = 0.0f, acc2 = 0.0f;  // this lane's share of the current (block, LP) run
  int run_lp = -1, run_slot = -1, run_go = 0;
  auto flush = [&]() {  // per warp: the warp's partial sums into its slot of the run
    if (run_lp >= 0 && run_go) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
        acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
      }
      if (lane == 0) ts.part[(size_t)run_slot * kWarps + warp] = make_float2(acc1, acc2);
    }
    acc1 = acc2 = 0.0f;
  };

  for (int i = 0; i < nmine; ++i) {
    const int s = i % kTileStages;
    const unsigned par = (unsigned)((i / kTileStages) & 1);
    const int gi = b + i * G;
    const TileItem it = ts.item[gi];
    unsigned char* st = smem + s * L::bytes;
    if (!mbar_wait(&bar_full[s], par)) {
      atomicExch(&fail, 1);
      break;
    }
    const StageMeta mt = meta[s];
    if (it.lp != run_lp) {
      flush();
      run_lp = it.lp;
      run_slot = gi;
      run_go = mt.go;
    }
    if (mt.go) {
      const int za = it.nb & ~7;
      int* col = reinterpret_cast<int*>(st + L::col);
      float* prb = reinterpret_cast<float*>(st + L::prb);
      const int* sp = reinterpret_cast<const int*>(st + L::ptr);
      const float2* xg = mt.cur ? d.x[0] : d.x[1];  // dual: x' of this attempt
      const float* yg = mt.cur ? d.y[1] : d.y[0];    // primal: current y
      // products of the staged nonzeros [q0, q1) (stage-relative), lanes strided,
      // eight gathers issued before any is used
      auto products = [&](int q0, int q1) {
        for (int q = q0 + lane; q < q1; q += 8 * 32) {
          if (DUAL) {
            float2 g[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int e = q + 32 * k;
              g[k] = e < q1 ? xg[col[e]] : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int e = q + 32 * k;
              if (e < q1) {
                const float v = stage_val<V>(st + L::val, e);
                col[e] = __float_as_int(v * g[k].x);
                prb[e] = v * g[k].y;
              }
            }
          } else {
            float g[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int e = q + 32 * k;
              g[k] = e < q1 ? yg[col[e]] : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const int e = q + 32 * k;
              if (e < q1) col[e] = __float_as_int(stage_val<V>(st + L::val, e) * g[k]);
            }
          }
        }
      };
      if (it.first < 0) {
        // tile: this warp's rows [w0, w1) of the item (stage-relative row w0 - r0)
        const int nr = it.r1 - it.r0;
        const int w0 = 32 * warp, w1 = min(nr, w0 + 32);
        if (w0 < w1) {
          const int po = it.r0 & 3;
          products(sp[po + w0] - za, sp[po + w1] - za);
          __syncwarp();
          const int t = w0 + lane;
          if (t < w1) {
            const int r = it.r0 + t;
            const int p0 = sp[po + t] - za, p1 = sp[po + t + 1] - za;
            float a = 0.0f, c2 = 0.0f;
            for (int p = p0; p < p1; ++p) {
              a += __int_as_float(col[p]);
              if (DUAL) c2 += prb[p];
            }
            const int k4 = po + t;
            const float* R0 = reinterpret_cast<const float*>(st + L::r0);
            const float* R1 = reinterpret_cast<const float*>(st + L::r1);
            const float* R2 = reinterpret_cast<const float*>(st + L::r2);
            const float* R3 = reinterpret_cast<const float*>(st + L::r3);
            const float* R4 = reinterpret_cast<const float*>(st + L::r4);
            if (DUAL) {
              const unsigned char* kinds = st + L::r5;
              const float2 tm = dual_row<IMPLICIT>(a, c2, R0[k4], IMPLICIT ? R1[k4] : 1.0f,
                                                   kinds[(it.r0 & 15) + t], R2[k4],
                                                   mt.pw != 0.0f ? R4[k4] : 0.0f, mt.step, mt.pw,
                                                   mt.cur ? d.y[0] : d.y[1], d.sum_y, r);
              acc1 += tm.x;
              acc2 += tm.y;
            } else {
              const float2* xs = reinterpret_cast<const float2*>(st + L::r5);
              acc1 += primal_row<IMPLICIT>(a, R0[k4], R1[k4], R2[k4], IMPLICIT ? R3[k4] : 1.0f,
                                           xs[(it.r0 & 1) + t].x, mt.pw != 0.0f ? R4[k4] : 0.0f,
                                           mt.step, mt.pw, mt.cur ? d.x[0] : d.x[1], d.sum_x, r);
            }
          }
        }
      } else {
        // slice: this warp's part of the nonzeros, then the eight parts in warp order
        const int o = it.nb - za, nz = it.ne - it.nb;
        const int part = ((nz + kWarps - 1) / kWarps + 31) & ~31;
        const int q0 = o + min(nz, warp * part), q1 = o + min(nz, (warp + 1) * part);
        products(q0, q1);
        __syncwarp();
        float a = 0.0f, c2 = 0.0f;
        for (int q = q0 + lane; q < q1; q += 32) {
          a += __int_as_float(col[q]);
          if (DUAL) c2 += prb[q];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, off);
          c2 += __shfl_xor_sync(0xffffffffu, c2, off);
        }
        int fin = 0;
        if (lane == 0) {
          slice_part[s][warp] = make_float2(a, c2);
          __threadfence_block();
          if (atomicAdd(&slice_done[s], 1) == kWarps - 1) {  // the last part: the slice's sum
            __threadfence_block();
            slice_done[s] = 0;
            float sa = 0.0f, sb = 0.0f;
            for (int k = 0; k < kWarps; ++k) {
              const float2 pv = slice_part[s][k];
              sa += pv.x;
              sb += pv.y;
            }
            ts.rowpart[gi] = make_float2(sa, sb);
            __threadfence();
            fin = atomicAdd(&ts.ticket[it.first], 1) == it.nsl - 1;
          }
        }
        fin = __shfl_sync(0xffffffffu, fin, 0);
        if (fin) {  // the last slice: the warp adds the slices' partials, lane 0 finishes the row
          __threadfence();
          float ra = 0.0f, rb = 0.0f;
          for (int k = lane; k < it.nsl; k += 32) {
            const float2 pv = __ldcg(ts.rowpart + it.first + k);
            ra += pv.x;
            rb += pv.y;
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            ra += __shfl_xor_sync(0xffffffffu, ra, off);
            rb += __shfl_xor_sync(0xffffffffu, rb, off);
          }
          if (lane == 0) {
            const int r = it.r0;
            if (DUAL) {
              const float* y = mt.cur ? d.y[1] : d.y[0];
              ts.lterm[it.lid] = dual_row<IMPLICIT>(
                  ra, rb, d.q[r], IMPLICIT ? d.sw[r] : 1.0f, d.row_kind[r], y[r],
                  mt.pw != 0.0f ? d.sum_y[r] : 0.0f, mt.step, mt.pw, mt.cur ? d.y[0] : d.y[1],
                  d.sum_y, r);
            } else {
              const float2* x = mt.cur ? d.x[1] : d.x[0];
              const float tm = primal_row<IMPLICIT>(
                  ra, d.c[r], d.l[r], d.u[r], IMPLICIT ? d.tw[r] : 1.0f, x[r].x,
                  mt.pw != 0.0f ? d.sum_x[r] : 0.0f, mt.step, mt.pw, mt.cur ? d.x[0] : d.x[1],
                  d.sum_x, r);
              ts.lterm[it.lid] = make_float2(tm, 0.0f);
            }
            ts.ticket[it.first] = 0;  // ready for the next launch
          }
        }
      }
    }
    // release the stage; the warp that releases it last requests its next item
    __syncwarp();
    if (lane == 0) {
      fence_proxy_async_smem();
      __threadfence_block();
      if (atomicAdd(&released[s], 1) == kWarps - 1) {
        __threadfence_block();
        released[s] = 0;
        if (i + kTileStages < nmine) {
          const TileItem nx = ts.item[gi + kTileStages * G];
          issue_const<V, DUAL, IMPLICIT>(st, nx, d, &bar_full[s]);
          meta[s] = item_meta<V, DUAL>(d, nx.lp);
          issue_iter<V, DUAL>(st, nx, d, meta[s], &bar_full[s]);
          issued[s] += 1;
        }
      }
    }
  }
  flush();
  // a stage never completed: record it; wait (bounded) for the copies still in flight
  // into the stages of items not consumed before the block exits
  __syncthreads();
  if (fail && tid == 0) {
    for (int s2 = 0; s2 < kTileStages; ++s2)
      if (issued[s2] > 0) (void)mbar_wait(&bar_full[s2], (unsigned)((issued[s2] - 1) & 1));
    for (int k = 0; k < d.count; ++k) atomicExch(&d.st[k].status, kStatusWaitFailed);
  }
}

}  // namespace pdlp
