// Bulk stream-collide through TMA: the hot kernel of the refined step.
//
// A tile is a run of 128 nodes along x at one (y, z).  For each of the 27
// populations the tile pulls one row segment, shifted by -c_i; rows are
// fetched with cp.async.bulk.tensor (TMA) as boxes [x0 - H, x0 + 128 + H)
// (H elements = 16 bytes, the start alignment TMA requires), so every shift
// of -1, 0, +1 along x is a fixed offset into the same shared-memory row.
// The three populations with the same (c_y, c_z) read the same source row
// of their planes, so one box of three rows (populations 3j .. 3j + 2)
// brings them: 9 loads per tile.  The post-collision tile is written to a
// shared-memory output stage and stored back by TMA, one box of 27 rows x 32
// nodes per warp.
//
// Warp roles: one thread of warp 4 is the producer -- it waits until a ring
// stage is free (mbarrier "empty"), posts the expected byte count and issues the
// 9 three-row loads of the next tile; warps 0-3 are consumers -- they wait for the
// stage (mbarrier "full"), read their 27 values, release the stage, collide,
// write their 32-node segment of the 27 output rows to shared memory and one
// lane stores it back with one TMA store, so consumer warps never wait for each
// other.  TMA instructions are issued by single threads: with per-lane operands
// the compiler would serialise them lane by lane.  Persistent CTAs walk a list
// of tiles whose rows pull by one rule per source row: from the neighbour row
// (wrapping only on spanned axes), or, beyond a wall across y or z, by
// bounce-back from the tile's own row.  Inlet and outlet rows and interface
// tiles take this path too: the inlet node keeps its populations, the outlet
// node pulls its c_x = -1 populations from itself, and nodes not updated in
// the substep are overwritten and rewritten later in the instant by the
// coupling.  Updated nodes whose pull the row rule cannot express (solid
// neighbours, walls across x) are recomputed afterwards from a fix-up list
// (k_sc_nodes); only tiles the row rule cannot serve at all go to k_sc_tiles,
// which pulls node by node.
//
// Waits suspend in hardware (mbarrier try_wait with a time hint) instead of
// spinning, so a waiting producer takes no issue slots from the consumers.
// Waits are bounded: a stage that does not arrive within the batch's bound
// (about a second unless the host sets it lower) sets bit 1 of the status
// word; the CTA then waits (with the full bound) for the copies it may have in
// flight and returns.
#pragma once
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "../../include/lbm.h"
#include "collide.cuh"
#include "device.cuh"
#include "kernels.h"
#include "warp.cuh"

namespace lbmk {

// Kernel variants the autotuner picks from: load stages DI, the CTAs per SM
// the register allocation aims for (MINB) and the tile shape, BX nodes along
// x.  Rows narrower than 128 nodes leave consumer warps of a 128-node tile
// idle; 64-node tiles (two consumer warps, from the halves of the 128-node
// tile list) keep them busy at more CTAs per SM.  Results do not depend on the
// variant.
template <typename S>
struct TmaVariants {
  static constexpr int N = 3;
  static constexpr int DI[N] = {sizeof(S) == 8 ? 2 : 3, sizeof(S) == 8 ? 1 : 2, 2};
  static constexpr int MINB[N] = {1, sizeof(S) == 8 ? 3 : 4, sizeof(S) == 8 ? 4 : 6};
  static constexpr int BX[N] = {128, 128, 64};
};

template <typename S, int DI_ = TmaVariants<S>::DI[0], int BX_ = 128>
struct TmaCfg {
  static_assert(BX_ == 64 || BX_ == 128, "tile shapes");
  static constexpr int BX = BX_;                                        // nodes per tile
  static constexpr int NCW = BX / 32;                                   // consumer warps
  static constexpr int H = 16 / (int)sizeof(S);                         // halo, elements
  static constexpr int W = BX + 2 * H;                                  // load box width, elements
  static constexpr int GROUP = (3 * W * (int)sizeof(S) + 127) / 128 * 128;  // bytes per three-row box
  static constexpr int OSEG = 32;                                       // nodes per warp segment
  static constexpr int OSEGB = (27 * OSEG * (int)sizeof(S) + 127) / 128 * 128;  // bytes per [27][32] segment
  static constexpr int SIDE = 128;                                      // one 16-byte wrap box, padded
  static constexpr int STAGE = 9 * GROUP + 18 * SIDE;                   // rows + 2 x 9 wrap boxes
  static constexpr int OSTAGE = NCW * OSEGB;                            // [warp][population][32 nodes]
  static constexpr uint32_t TX = 27u * W * (uint32_t)sizeof(S);        // bytes of the 27 row loads
  static constexpr uint32_t TXW = 9u * 16u;                             // bytes of 9 wrap boxes
  static constexpr int DI = DI_;                                        // load stages
  static constexpr int DO = 1;                                          // store stages
  static constexpr int SMEM = DI * STAGE + DO * OSTAGE + 128;           // + slack for 128-byte alignment
  static constexpr int THREADS = BX + 32;                               // consumer warps + 1 producer
};

template <typename S>
struct SCvt;
template <>
struct SCvt<double> {
  static __device__ __forceinline__ double to(double v) { return v; }
};
template <>
struct SCvt<float> {
  static __device__ __forceinline__ float to(float v) { return v; }
};
template <>
struct SCvt<__half> {
  static __device__ __forceinline__ float to(__half v) { return __half2float(v); }
};
template <>
struct SCvt<__nv_bfloat16> {
  static __device__ __forceinline__ float to(__nv_bfloat16 v) { return __bfloat162float(v); }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// try_wait that may suspend the thread for up to ns nanoseconds (woken early
// when the phase completes).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

// Non-blocking test of an mbarrier phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase: up to `sleeps` suspensions of at most
// 0.5 us each (kWaitSleeps: about a second); sleeps = 0 tests once without
// waiting.
constexpr int kWaitSleeps = 1 << 21;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int sleeps = kWaitSleeps) {
  if (sleeps <= 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  for (int it = 0; it < sleeps; ++it)
    if (mbar_try_wait_sleep(bar, parity, 500u)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                             int i) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(i), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_store_row(const CUtensorMap* map, const void* src, int x, int y, int z, int i) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(i), "r"(smem_u32(src))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_row(const CUtensorMap* map, int x, int y, int z, int i) {
  asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(i)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int wrap_axis(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// tile list entries: x-tile | y << 16 | z << 32 | bounce mask << 48 | flags << 57
// (flag 1: the row's first node is a fixed inlet node; flag 2: its last node
// is the zero-gradient outlet)
__device__ __forceinline__ void tile_xyz(unsigned long long t, int& tx, int& y, int& z) {
  tx = (int)(t & 0xffffu);
  y = (int)((t >> 16) & 0xffffu);
  z = (int)((t >> 32) & 0xffffu);
}
__device__ __forceinline__ int tile_bounce(unsigned long long t) { return (int)((t >> 48) & 0x1ffu); }
__device__ __forceinline__ int tile_flags(unsigned long long t) { return (int)((t >> 57) & 3u); }

// Shared-memory row of population i in a load stage (elements): group i / 3,
// row i % 3 of the three-row box.
template <typename S, int BX = 128>
__device__ __forceinline__ constexpr int row_base(int i) {
  using C = TmaCfg<S, TmaVariants<S>::DI[0], BX>;
  return (i / 3) * (C::GROUP / (int)sizeof(S)) + (i % 3) * C::W;
}

// Walls across y or z: when the source row j = (c_y + 1) + 3 (c_z + 1) of a
// tile lies beyond a wall (bit j of the tile's bounce mask), its three
// populations i = 3j + k bounce back, f_i(x) = f'_{26-i}(x) at the same node:
// the stage slot of row j then holds the box of populations 3(8 - j) .. 3(8 - j) + 2
// from the tile's own row, and population 3j + k reads its row 2 - k unshifted.
//
// Inflow along x: a fixed inlet node (x = 0) keeps its populations -- its
// thread reads them from global memory and writes them back unchanged -- and
// the outlet node (x = dim - 1) pulls its c_x = -1 populations from itself
// along x (zero gradient), which the stage holds unshifted.
//
// Periodic x: the first tile of a row needs, for the 9 populations with
// c_x = +1 (i = 3j + 2), the element at x = dim - 1; the last tile, for the 9
// with c_x = -1 (i = 3j), the element at x = 0.  Both come as 16-byte boxes
// (map_wrap) into side slots after the 27 rows of the stage: slot j holds
// [dim - H, dim) of population 3j + 2, slot 9 + j holds [0, H) of population 3j.
// Every TMA destination in shared memory starts on a 128-byte boundary.
//
// Batching: one launch sweeps the TMA tiles of every patch stepped at an
// instant (patches of uneven sizes on several levels), as the concatenation of
// their tile lists; each tile carries its patch's tensor maps, geometry,
// relaxation and force.
constexpr int kTmaBatch = 8;  // patches per launch
constexpr long long kWarpNodes = 152 * 4 * 128;  // fix-up lists up to this size go one warp per node

template <typename S, typename R>
struct TmaPatch {
  CUtensorMap map_in, map_out, map_wrap;
  PatchDev p;
  const S* fin;                          // current populations (fixed inlet nodes are copied from it)
  const unsigned long long* tiles;       // this patch's tile list
  int tile0, ntiles;                     // its range in the concatenated tile index
  R beta, du[3];
};

template <typename S, typename R>
struct TmaBatch {
  TmaPatch<S, R> e[kTmaBatch];
  int n, ntiles, lbgk;
  int wait_sleeps;  // bound of the consumers' waits for a loaded stage (mbar_wait_bounded)
  int* status;
};

template <typename S, typename R>
__device__ __forceinline__ int batch_entry(const TmaBatch<S, R>& b, int t) {
  int e = 0;
#pragma unroll
  for (int q = 1; q < kTmaBatch; ++q)
    if (q < b.n && t >= b.e[q].tile0) e = q;
  return e;
}

// MINB: CTAs per SM the register allocation aims for (launch bounds); BX:
// nodes per tile (BX / 32 consumer warps, then the producer warp).
template <typename S, typename R, int FM, int DI, int MINB, int BX = 128>
__global__ void __launch_bounds__(BX + 32, MINB) k_sc_tma(const __grid_constant__ TmaBatch<S, R> b) {
  using C = TmaCfg<S, DI, BX>;
  const int ntiles = b.ntiles;
  int* status = b.status;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* ostage = smem + C::DI * C::STAGE;
  __shared__ __align__(8) uint64_t full[C::DI], empty[C::DI];
  __shared__ int4 tile_at[C::DI];  // tile coordinates of each stage, published with its mbarrier
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nmine = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  if (tid == 0) {
    for (int s = 0; s < C::DI; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], C::NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == C::NCW) {
    // ---------------- producer (one thread: TMA operands stay warp-uniform) ----------------
    if (lane != 0) return;
    for (int q = 0; q < b.n; ++q) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&b.e[q].map_in)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&b.e[q].map_out)) : "memory");
    }
    for (int k = 0; k < nmine; ++k) {
      const int s = k % C::DI;
      if (k >= C::DI && !mbar_wait_bounded(&empty[s], (uint32_t)((k / C::DI) - 1) & 1u)) {
        atomicOr(status, 2);
        return;  // consumers time out on the stages never filled
      }
      const int t = (int)blockIdx.x + k * (int)gridDim.x;
      const int ei = batch_entry(b, t);
      const TmaPatch<S, R>& E = b.e[ei];
      const PatchDev& p = E.p;
      int tx, ty, tz;
      const unsigned long long te = E.tiles[t - E.tile0];
      tile_xyz(te, tx, ty, tz);
      const int bm = tile_bounce(te);
      const int fl = tile_flags(te);
      const bool first = p.span[0] && tx == 0;
      const bool last = p.span[0] && (tx + 1) * C::BX >= p.dim[0];
      tile_at[s] = make_int4(tx, ty, tz, bm | (fl << 9) | (ei << 11));
      const uint32_t txw = 16u * (uint32_t)(9 - __popc(bm));  // wrap boxes of the rows not bounced
      mbar_expect_tx(&full[s], C::TX + (first ? txw : 0u) + (last ? txw : 0u));
      unsigned char* stage = smem + s * C::STAGE;
      unsigned char* side = stage + 9 * C::GROUP;
      const int x0 = tx * C::BX - C::H;
#pragma unroll 1
      for (int cz = 0; cz < 3; ++cz) {
        const int sz = wrap_axis(tz - (cz - 1), p.dim[2]);
#pragma unroll 1
        for (int cy = 0; cy < 3; ++cy) {
          const int sy = wrap_axis(ty - (cy - 1), p.dim[1]);
          const int j = 3 * cz + cy;  // populations 3j, 3j + 1, 3j + 2 share this source row
          if ((bm >> j) & 1) {
            tma_load_row(stage + j * C::GROUP, &E.map_in, &full[s], x0, ty, tz, 3 * (8 - j));
            continue;
          }
          tma_load_row(stage + j * C::GROUP, &E.map_in, &full[s], x0, sy, sz, 3 * j);
          if (first) tma_load_row(side + j * C::SIDE, &E.map_wrap, &full[s], p.dim[0] - C::H, sy, sz, 3 * j + 2);
          if (last) tma_load_row(side + (9 + j) * C::SIDE, &E.map_wrap, &full[s], 0, sy, sz, 3 * j);
        }
      }
    }
    return;
  }

  // ---------------- consumers (warps 0 .. NCW - 1) ----------------
  for (int k = 0; k < nmine; ++k) {
    const int s = k % C::DI;
    const bool ok = mbar_wait_bounded(&full[s], (uint32_t)(k / C::DI) & 1u, b.wait_sleeps);
    if (!ok) {
      // stage not arrived in time: flag, wait (full bound) for the loads that
      // may still be in flight, this stage's included, drain stores, leave
      if (lane == 0) atomicOr(status, 2);
      for (int j = k; j < nmine && j < k + C::DI; ++j) mbar_wait_bounded(&full[j % C::DI], (uint32_t)(j / C::DI) & 1u);
      if (lane == 0) bulk_wait_all();
      return;
    }
    const int4 tc = tile_at[s];
    const int tx = tc.x, y = tc.y, z = tc.z, bm = tc.w & 0x1ff, fl = (tc.w >> 9) & 3;
    const TmaPatch<S, R>& E = b.e[tc.w >> 11];
    const PatchDev& p = E.p;
    const int x = tx * C::BX + tid;
    const S* st = reinterpret_cast<const S*>(smem + s * C::STAGE);
    R f[27];
    if (bm == 0) {
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = SCvt<S>::to(st[row_base<S, BX>(i) + C::H + tid - CX(i)]);
      });
    } else {
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const bool b = (bm >> (i / 3)) & 1;
        f[i] = SCvt<S>::to(st[b ? row_base<S, BX>(3 * (i / 3) + 2 - i % 3) + C::H + tid
                                : row_base<S, BX>(i) + C::H + tid - CX(i)]);
      });
    }
    if (p.span[0] && (x == 0 || x == p.dim[0] - 1)) {
      // periodic wrap along x from the side slots (rows not bounced)
      const S* side = reinterpret_cast<const S*>(smem + s * C::STAGE + 9 * C::GROUP);
      const bool lo = x == 0;
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const bool b = (bm >> (i / 3)) & 1;
        if (!b && lo && CX(i) == 1) f[i] = SCvt<S>::to(side[(i / 3) * (C::SIDE / (int)sizeof(S)) + C::H - 1]);
        if (!b && !lo && CX(i) == -1) f[i] = SCvt<S>::to(side[(9 + i / 3) * (C::SIDE / (int)sizeof(S))]);
      });
    }
    bool fixed = false;
    if (fl) {
      if ((fl & 2) && x == p.dim[0] - 1) {
        // zero-gradient outlet: c_x = -1 populations from the node itself along x
        unroll<27>([&](auto I) {
          constexpr int i = decltype(I)::value;
          if (CX(i) == -1 && !((bm >> (i / 3)) & 1)) f[i] = SCvt<S>::to(st[row_base<S, BX>(i) + C::H + tid]);
        });
      }
      if ((fl & 1) && x == 0) {
        fixed = true;
        const long long own = node_index(p, 0, y, z);
        unroll<27>([&](auto I) {
          constexpr int i = decltype(I)::value;
          f[i] = Stor<S>::ld(E.fin + (long long)i * p.plane + own);
        });
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with stage s
    if (x < p.dim[0] && !fixed) kbc_collide<R, FM>(f, E.beta, E.du[0], E.du[1], E.du[2], b.lbgk != 0);
    // this warp's output segment in stage o: wait until the stores that last
    // used it have read it, fill it, store it
    const int o = k % C::DO;
    if (lane == 0) bulk_wait_read<C::DO - 1>();
    __syncwarp();
    unsigned char* seg = ostage + o * C::OSTAGE + warp * C::OSEGB;
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Stor<S>::st(reinterpret_cast<S*>(seg) + i * C::OSEG + lane, f[i]);
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      tma_store_row(&E.map_out, seg, tx * C::BX + warp * C::OSEG, y, z, 0);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// The tile pass on node pairs (FP32 arithmetic, any FP32 or 16-bit storage).
// Same tiles, stage layout and row rule as k_sc_tma; a consumer thread takes
// two neighbouring nodes x, x + 1 of its warp's 64-node half of a tile and
// collides them together with the packed FP32x2 instructions (F2), so one
// instruction stream serves two nodes.  Results equal k_sc_tma's bit for bit
// (collide.cuh).  A pair's populations with c_x = 0 and the bounced ones sit
// at an even offset of the stage row and load as one 8-byte (4-byte for
// 16-bit) word; the others load as two elements.  Each warp stores its half
// tile as two [27][32] boxes.
template <typename S>
struct Pair;
template <>
struct Pair<float> {
  static __device__ __forceinline__ F2 ld2(const float* p) {  // p 8-byte aligned
    return F2(*reinterpret_cast<const float2*>(p));
  }
  static __device__ __forceinline__ void st2(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <>
struct Pair<__half> {
  static __device__ __forceinline__ F2 ld2(const __half* p) {
    return F2(__half22float2(*reinterpret_cast<const __half2*>(p)));
  }
  static __device__ __forceinline__ void st2(__half* p, F2 v) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.v.x, v.v.y);
  }
};
template <>
struct Pair<__nv_bfloat16> {
  static __device__ __forceinline__ F2 ld2(const __nv_bfloat16* p) {
    return F2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  static __device__ __forceinline__ void st2(__nv_bfloat16* p, F2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.v.x, v.v.y);
  }
};

// Loads of one tile into a stage (the producer's part of k_sc_tma, shared by
// k_sc_tma2, where consumer threads issue them): 9 three-row boxes, the
// bounce rule, the x-periodic wrap boxes; records the tile in tile_at.
template <typename S, int DI>
__device__ __forceinline__ void issue_tile(const TmaBatch<S, float>& b, int t, unsigned char* stage,
                                           uint64_t* full, int4* tile_at) {
  using C = TmaCfg<S, DI>;
  const int ei = batch_entry(b, t);
  const TmaPatch<S, float>& E = b.e[ei];
  const PatchDev& p = E.p;
  int tx, ty, tz;
  const unsigned long long te = E.tiles[t - E.tile0];
  tile_xyz(te, tx, ty, tz);
  const int bm = tile_bounce(te);
  const int fl = tile_flags(te);
  const bool first = p.span[0] && tx == 0;
  const bool last = p.span[0] && (tx + 1) * C::BX >= p.dim[0];
  *tile_at = make_int4(tx, ty, tz, bm | (fl << 9) | (ei << 11));
  const uint32_t txw = 16u * (uint32_t)(9 - __popc(bm));  // wrap boxes of the rows not bounced
  mbar_expect_tx(full, C::TX + (first ? txw : 0u) + (last ? txw : 0u));
  unsigned char* side = stage + 9 * C::GROUP;
  const int x0 = tx * C::BX - C::H;
#pragma unroll 1
  for (int j = 0; j < 9; ++j) {
    if ((bm >> j) & 1) {
      tma_load_row(stage + j * C::GROUP, &E.map_in, full, x0, ty, tz, 3 * (8 - j));
      continue;
    }
    const int sy = wrap_axis(ty - (j % 3 - 1), p.dim[1]);
    const int sz = wrap_axis(tz - (j / 3 - 1), p.dim[2]);
    tma_load_row(stage + j * C::GROUP, &E.map_in, full, x0, sy, sz, 3 * j);
    if (first) tma_load_row(side + j * C::SIDE, &E.map_wrap, full, p.dim[0] - C::H, sy, sz, 3 * j + 2);
    if (last) tma_load_row(side + (9 + j) * C::SIDE, &E.map_wrap, full, 0, sy, sz, 3 * j);
  }
}

// No producer warp: NP pairs of consumer warps take alternate tiles of the
// CTA's sequence from a ring of DI stages (DI a multiple of NP, so each pair
// cycles through DI / NP stages of its own).  Thread 0 loads the first DI
// tiles; after a pair has read tile k (named barrier of its 64 threads), its
// first thread loads tile k + DI into the same stage.  Without the producer
// a CTA has NP * 2 warps, so two CTAs of two pairs fit the register file at
// up to 255 registers a thread: two consumer warps per SM sub-partition.
template <typename S, int FM, int DI, int NP, int MINB>
__global__ void __launch_bounds__(NP * 64, MINB) k_sc_tma2(const __grid_constant__ TmaBatch<S, float> b) {
  static_assert(DI % NP == 0, "each pair owns DI / NP stages");
  using C = TmaCfg<S, DI>;
  const int ntiles = b.ntiles;
  int* status = b.status;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* ostage = smem + DI * C::STAGE;
  __shared__ __align__(8) uint64_t full[DI];
  __shared__ int4 tile_at[DI];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nmine = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  if (tid == 0) {
    for (int s = 0; s < DI; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < b.n; ++q) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&b.e[q].map_in)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&b.e[q].map_out)) : "memory");
    }
    for (int k = 0; k < nmine && k < DI; ++k)
      issue_tile<S, DI>(b, (int)blockIdx.x + k * (int)gridDim.x, smem + k * C::STAGE, &full[k], &tile_at[k]);
  }
  __syncthreads();

  const int cp = warp >> 1, h = warp & 1;
  const bool leader = h == 0 && lane == 0;
  const int e0 = 64 * h + 2 * lane;  // offset of the thread's first node in the tile
  unsigned char* myseg = ostage + warp * 2 * C::OSEGB;
  for (int k = cp; k < nmine; k += NP) {
    const int s = k % DI;
    if (!mbar_wait_bounded(&full[s], (uint32_t)(k / DI) & 1u, b.wait_sleeps)) {
      // not arrived in time: flag, wait (full bound) for the loads that may
      // still be in flight, this stage's included, drain stores, leave
      if (lane == 0) atomicOr(status, 2);
      for (int j = k; j < nmine && j < k + DI; j += NP) mbar_wait_bounded(&full[j % DI], (uint32_t)(j / DI) & 1u);
      if (lane == 0) bulk_wait_all();
      return;
    }
    const int4 tc = tile_at[s];
    const int tx = tc.x, y = tc.y, z = tc.z, bm = tc.w & 0x1ff, fl = (tc.w >> 9) & 3;
    const TmaPatch<S, float>& E = b.e[tc.w >> 11];
    const PatchDev& p = E.p;
    const int xa = tx * C::BX + e0;  // the pair's nodes: xa, xa + 1
    const S* st = reinterpret_cast<const S*>(smem + s * C::STAGE);
    F2 f[27];
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      constexpr int cx = CX(i);
      if ((bm >> (i / 3)) & 1) {
        f[i] = Pair<S>::ld2(st + row_base<S>(3 * (i / 3) + 2 - i % 3) + C::H + e0);
      } else if constexpr (cx == 0) {
        f[i] = Pair<S>::ld2(st + row_base<S>(i) + C::H + e0);
      } else {
        const S* r = st + row_base<S>(i) + C::H + e0 - cx;
        f[i] = F2(SCvt<S>::to(r[0]), SCvt<S>::to(r[1]));
      }
    });
    // rare nodes, lane by lane: x-periodic wrap, outlet, tail beyond the row
    const bool lo_edge = xa == 0, hi_a = xa == p.dim[0] - 1, hi_b = xa + 1 == p.dim[0] - 1;
    if (p.span[0] && (lo_edge || hi_a || hi_b)) {
      const S* side = reinterpret_cast<const S*>(smem + s * C::STAGE + 9 * C::GROUP);
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if ((bm >> (i / 3)) & 1) return;
        if constexpr (CX(i) == 1) {
          if (lo_edge) f[i].v.x = SCvt<S>::to(side[(i / 3) * (C::SIDE / (int)sizeof(S)) + C::H - 1]);
        }
        if constexpr (CX(i) == -1) {
          const float w = SCvt<S>::to(side[(9 + i / 3) * (C::SIDE / (int)sizeof(S))]);
          if (hi_a) f[i].v.x = w;
          if (hi_b) f[i].v.y = w;
        }
      });
    }
    if ((fl & 2) && (hi_a || hi_b)) {
      // zero-gradient outlet: c_x = -1 populations from the node itself along x
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (CX(i) == -1) {
          if (!((bm >> (i / 3)) & 1)) {
            const S* r = st + row_base<S>(i) + C::H + e0;
            if (hi_a) f[i].v.x = SCvt<S>::to(r[0]);
            if (hi_b) f[i].v.y = SCvt<S>::to(r[1]);
          }
        }
      });
    }
    if (xa + 1 >= p.dim[0]) {
      // beyond the row (storage padding): the rest state, so that the
      // arithmetic stays finite; TMA stores it into the padding
      const bool out_a = xa >= p.dim[0];
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (out_a) f[i].v.x = 0.0f;
        f[i].v.y = 0.0f;
      });
    }
    // both warps of the pair have read stage s: its leader loads the pair's
    // tile k + DI into it
    asm volatile("bar.sync %0, 64;" ::"r"(1 + cp) : "memory");
    if (leader && k + DI < nmine)
      issue_tile<S, DI>(b, (int)blockIdx.x + (k + DI) * (int)gridDim.x, smem + s * C::STAGE, &full[s], &tile_at[s]);
    {
      F2 rho_t, rho, ux, uy, uz;
      macro_v<F2>(f, rho_t, rho, ux, uy, uz);
      kbc_collide_v<F2, FM>(f, rho_t, rho, ux, uy, uz, F2(E.beta), F2(E.du[0]), F2(E.du[1]), F2(E.du[2]),
                            E.du[0] != 0.0f, E.du[1] != 0.0f, E.du[2] != 0.0f, b.lbgk != 0);
    }
    if ((fl & 1) && lo_edge) {
      // fixed inlet node: keeps its populations
      const long long own = node_index(p, 0, y, z);
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i].v.x = Stor<S>::ld(E.fin + (long long)i * p.plane + own);
      });
    }
    // this warp's two [27][32] output segments: wait until the stores that
    // last used them have read them, fill, store
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
    S* seg = reinterpret_cast<S*>(myseg + (lane >> 4) * C::OSEGB) + ((2 * lane) & 31);
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      Pair<S>::st2(seg + i * C::OSEG, f[i]);
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      tma_store_row(&E.map_out, myseg, tx * C::BX + 64 * h, y, z, 0);
      tma_store_row(&E.map_out, myseg + C::OSEGB, tx * C::BX + 64 * h + 32, y, z, 0);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
}

// Mixed tiles: node-by-node pull (walls, solids, outlet, interface layers).
template <typename S, typename R, int FM>
__global__ void __launch_bounds__(128) k_sc_tiles(PatchDev p, const S* __restrict__ fin, S* __restrict__ fout,
                                                  const uint32_t* __restrict__ tiles, int ntx, R beta, R dux, R duy,
                                                  R duz, int odd, int lbgk, int* status) {
  const uint32_t t = tiles[blockIdx.x];
  const int x = (int)(t % (uint32_t)ntx) * 128 + threadIdx.x;
  const int y = (int)((t / (uint32_t)ntx) % (uint32_t)p.dim[1]);
  const int z = (int)(t / ((uint32_t)ntx * (uint32_t)p.dim[1]));
  if (x >= p.dim[0]) return;
  const long long own = node_index(p, x, y, z);
  const uint8_t ty = p.type[own];
  if (!(ty == T_BULK || ty == T_BC || (ty == T_D1 && odd))) return;
  R f[27];
  if (ty == T_BULK) pull_bulk<S, R>(p, fin, x, y, z, f);
  else pull_generic<S, R, true>(p, fin, x, y, z, f, status);
  kbc_collide<R, FM>(f, beta, dux, duy, duz, lbgk != 0);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Stor<S>::st(fout + (long long)i * p.plane + own, f[i]);
  });
}

// Fix-up nodes: updated nodes of TMA tiles whose pulls the row rule does not
// give (solid neighbours, x walls), recomputed node by node after the tile pass.
template <typename S, typename R, int FM>
__global__ void __launch_bounds__(128) k_sc_nodes(PatchDev p, const S* __restrict__ fin, S* __restrict__ fout,
                                                  const uint32_t* __restrict__ nodes, long long n, R beta, R dux,
                                                  R duy, R duz, int lbgk, int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const long long own = nodes[k];
  const int x = (int)(own % p.nxp), y = (int)((own / p.nxp) % p.dim[1]);
  const int z = (int)(own / ((long long)p.nxp * p.dim[1]));
  R f[27];
  pull_generic<S, R, true>(p, fin, x, y, z, f, status);
  kbc_collide<R, FM>(f, beta, dux, duy, duz, lbgk != 0);
  unroll<27>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Stor<S>::st(fout + (long long)i * p.plane + own, f[i]);
  });
}

// Fix-up nodes, one warp per node (warp.cuh): for the few thousand fix-up
// nodes around a solid body, where the few warps of a thread-per-node launch
// would wait on the instruction fetch of its long unrolled code.
template <typename S, typename R>
__global__ void __launch_bounds__(128) k_sc_nodes_w(PatchDev p, const S* __restrict__ fin, S* __restrict__ fout,
                                                    const uint32_t* __restrict__ nodes, long long n, R beta, R dux,
                                                    R duy, R duz, int lbgk, int* status) {
  const long long k = warp_id();
  if (k >= n) return;  // whole warp
  const Lane d = lane_dir();
  const long long own = nodes[k];
  const int x = (int)(own % p.nxp), y = (int)((own / p.nxp) % p.dim[1]);
  const int z = (int)(own / ((long long)p.nxp * p.dim[1]));
  bool bad = false;
  const R f = d.on ? wpull_generic<S, R>(p, fin, x, y, z, d, bad) : R(0);
  if (__any_sync(kFullMask, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1);
  const R fo = wkbc_collide<R>(f, d, beta, dux, duy, duz, lbgk != 0);
  if (d.on) Stor<S>::st(fout + (long long)d.i * p.plane + own, fo);
}

template <typename S, typename R, int FM, int V>
cudaError_t launch_tma_v(const TmaBatch<S, R>& b, cudaStream_t st) {
  constexpr int DI = TmaVariants<S>::DI[V], MINB = TmaVariants<S>::MINB[V], BX = TmaVariants<S>::BX[V];
  using C = TmaCfg<S, DI, BX>;
  static int blocks_per_sm = -1, sms = 0;
  auto kern = k_sc_tma<S, R, FM, DI, MINB, BX>;
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, C::THREADS, C::SMEM);
    if (e) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int grid = std::min(b.ntiles, blocks_per_sm * sms);
  kern<<<grid, C::THREADS, C::SMEM, st>>>(b);
  return cudaGetLastError();
}

// Packed-pair variants (k_sc_tma2): load stages, consumer pairs, CTAs per SM.
struct Tma2Variant {
  int di, np, minb;
};
constexpr Tma2Variant kTma2[2] = {{4, 2, 3}, {2, 2, 3}};

template <typename S, int FM, int V>
cudaError_t launch_tma2_v(const TmaBatch<S, float>& b, cudaStream_t st) {
  constexpr int DI = kTma2[V].di, NP = kTma2[V].np, MINB = kTma2[V].minb;
  using C = TmaCfg<S, DI>;
  constexpr int THREADS = NP * 64;
  constexpr int SMEM = DI * C::STAGE + 2 * NP * 2 * C::OSEGB + 128;
  static int blocks_per_sm = -1, sms = 0;
  auto kern = k_sc_tma2<S, FM, DI, NP, MINB>;
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, THREADS, SMEM);
    if (e) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  const int grid = std::min(b.ntiles, blocks_per_sm * sms);
  kern<<<grid, THREADS, SMEM, st>>>(b);
  return cudaGetLastError();
}

// Variants: 0, 1 the scalar kernel on 128-node tiles; for FP32 arithmetic
// 2, 3 the node-pair kernel; last (2 for FP64, 4 otherwise) the scalar kernel
// on 64-node tiles, whose batch carries the half-tile lists and descriptors
// (sc_tma_tile_nodes).
template <typename S, typename R, int FM>
cudaError_t launch_tma_fm(const TmaBatch<S, R>& b, int variant, cudaStream_t st) {
  static_assert(TmaVariants<S>::N == 3 && TmaVariants<S>::BX[2] == 64, "variant dispatch");
  if constexpr (std::is_same<R, float>::value) {
    if (variant == 2) return launch_tma2_v<S, FM, 0>(b, st);
    if (variant == 3) return launch_tma2_v<S, FM, 1>(b, st);
    if (variant == 4) return launch_tma_v<S, R, FM, 2>(b, st);
  } else {
    if (variant == 2) return launch_tma_v<S, R, FM, 2>(b, st);
  }
  return variant == 1 ? launch_tma_v<S, R, FM, 1>(b, st) : launch_tma_v<S, R, FM, 0>(b, st);
}

// One launch over up to kTmaBatch patches (their force masks must agree).
template <typename S, typename R>
cudaError_t sc_tma_typed(const TmaLaunchPatch* ps, int n, int variant, int lbgk, int wait_sleeps, int* status,
                         cudaStream_t st) {
  TmaBatch<S, R> b;
  memset(&b, 0, sizeof b);
  b.lbgk = lbgk;
  b.wait_sleeps = wait_sleeps;
  b.status = status;
  int fm = 0;
  for (int q = 0; q < n; ++q) {
    if (ps[q].ntiles <= 0) continue;
    if (b.n == kTmaBatch) return cudaErrorInvalidValue;
    TmaPatch<S, R>& E = b.e[b.n++];
    memcpy(&E.map_in, ps[q].tmap_in, sizeof(CUtensorMap));
    memcpy(&E.map_out, ps[q].tmap_out, sizeof(CUtensorMap));
    memcpy(&E.map_wrap, ps[q].tmap_wrap, sizeof(CUtensorMap));
    E.p = ps[q].p;
    E.fin = (const S*)ps[q].fin;
    E.tiles = ps[q].tiles;
    E.tile0 = b.ntiles;
    E.ntiles = (int)ps[q].ntiles;
    E.beta = (R)ps[q].beta;
    for (int a = 0; a < 3; ++a) E.du[a] = (R)ps[q].F.du[a];
    b.ntiles += E.ntiles;
    fm |= ps[q].F.mask();
  }
  if (b.ntiles == 0) return cudaSuccess;
  switch (fm) {
    case 0:
      return launch_tma_fm<S, R, 0>(b, variant, st);
    case 1:
      return launch_tma_fm<S, R, 1>(b, variant, st);
    case 4:
      return launch_tma_fm<S, R, 4>(b, variant, st);
    default:
      return launch_tma_fm<S, R, 7>(b, variant, st);
  }
}

template <typename S, typename R>
cudaError_t sc_nodes_typed(const PatchDev& p, const void* fin, void* fout, const uint32_t* nodes, int64_t n,
                           double beta, const Force& F, int lbgk, int* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const R b = (R)beta, dx = (R)F.du[0], dy = (R)F.du[1], dz = (R)F.du[2];
  const unsigned grid = (unsigned)((n + 127) / 128);
  const S* in = (const S*)fin;
  S* out = (S*)fout;
  // up to this many nodes a thread per node leaves the SMs nearly empty
  // (fewer than four blocks of 128 per SM): one warp per node instead
  if (n <= kWarpNodes) {
    k_sc_nodes_w<S, R><<<(unsigned)((n + 3) / 4), 128, 0, st>>>(p, in, out, nodes, n, b, dx, dy, dz, lbgk, status);
    return cudaGetLastError();
  }
  switch (F.mask()) {
    case 0:
      k_sc_nodes<S, R, 0><<<grid, 128, 0, st>>>(p, in, out, nodes, n, b, dx, dy, dz, lbgk, status);
      break;
    case 1:
      k_sc_nodes<S, R, 1><<<grid, 128, 0, st>>>(p, in, out, nodes, n, b, dx, dy, dz, lbgk, status);
      break;
    case 4:
      k_sc_nodes<S, R, 4><<<grid, 128, 0, st>>>(p, in, out, nodes, n, b, dx, dy, dz, lbgk, status);
      break;
    default:
      k_sc_nodes<S, R, 7><<<grid, 128, 0, st>>>(p, in, out, nodes, n, b, dx, dy, dz, lbgk, status);
  }
  return cudaGetLastError();
}

template <typename S, typename R>
cudaError_t sc_tiles_typed(const PatchDev& p, const void* fin, void* fout, const uint32_t* tiles, int64_t ntiles,
                           int ntx, double beta, const Force& F, int odd, int lbgk, int* status, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const R b = (R)beta, dx = (R)F.du[0], dy = (R)F.du[1], dz = (R)F.du[2];
  const dim3 grid((unsigned)ntiles), block(128);
  const S* in = (const S*)fin;
  S* out = (S*)fout;
  switch (F.mask()) {
    case 0:
      k_sc_tiles<S, R, 0><<<grid, block, 0, st>>>(p, in, out, tiles, ntx, b, dx, dy, dz, odd, lbgk, status);
      break;
    case 1:
      k_sc_tiles<S, R, 1><<<grid, block, 0, st>>>(p, in, out, tiles, ntx, b, dx, dy, dz, odd, lbgk, status);
      break;
    case 4:
      k_sc_tiles<S, R, 4><<<grid, block, 0, st>>>(p, in, out, tiles, ntx, b, dx, dy, dz, odd, lbgk, status);
      break;
    default:
      k_sc_tiles<S, R, 7><<<grid, block, 0, st>>>(p, in, out, tiles, ntx, b, dx, dy, dz, odd, lbgk, status);
  }
  return cudaGetLastError();
}

// per-storage entry points, one translation unit each
#define LBM_SC_DECL(NAME)                                                                                        \
  cudaError_t sc_tma_##NAME(const TmaLaunchPatch* ps, int n, int variant, int lbgk, int wait_sleeps,           \
                            int* status, cudaStream_t st);                                                       \
  cudaError_t sc_tiles_##NAME(const PatchDev& p, const void* fin, void* fout, const uint32_t* tiles,             \
                              int64_t ntiles, int ntx, double beta, const Force& F, int odd, int lbgk,           \
                              int* status, cudaStream_t st);                                                     \
  cudaError_t sc_nodes_##NAME(const PatchDev& p, const void* fin, void* fout, const uint32_t* nodes, int64_t n,  \
                              double beta, const Force& F, int lbgk, int* status, cudaStream_t st);
LBM_SC_DECL(fp64)
LBM_SC_DECL(fp32)
LBM_SC_DECL(fp16)
LBM_SC_DECL(bf16)

#define LBM_SC_DEFINE(NAME, S, R)                                                                                \
  cudaError_t sc_tma_##NAME(const TmaLaunchPatch* ps, int n, int variant, int lbgk, int wait_sleeps,           \
                            int* status, cudaStream_t st) {                                                      \
    return sc_tma_typed<S, R>(ps, n, variant, lbgk, wait_sleeps, status, st);                                    \
  }                                                                                                              \
  cudaError_t sc_tiles_##NAME(const PatchDev& p, const void* fin, void* fout, const uint32_t* tiles,             \
                              int64_t ntiles, int ntx, double beta, const Force& F, int odd, int lbgk,           \
                              int* status, cudaStream_t st) {                                                    \
    return sc_tiles_typed<S, R>(p, fin, fout, tiles, ntiles, ntx, beta, F, odd, lbgk, status, st);               \
  }                                                                                                              \
  cudaError_t sc_nodes_##NAME(const PatchDev& p, const void* fin, void* fout, const uint32_t* nodes, int64_t n,  \
                              double beta, const Force& F, int lbgk, int* status, cudaStream_t st) {             \
    return sc_nodes_typed<S, R>(p, fin, fout, nodes, n, beta, F, lbgk, status, st);                              \
  }

}  // namespace lbmk
