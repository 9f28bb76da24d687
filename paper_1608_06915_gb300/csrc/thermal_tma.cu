// Thermal stream-collide through TMA: the tile pass of the two-population
// model, built like the isothermal one (sc_tma.cuh) with both sets staged.
//
// A tile is 128 nodes along x at one (y, z).  The producer thread loads, per
// tile, 9 three-row boxes of f and 9 of g (one box per source row (c_y, c_z),
// populations 3j .. 3j + 2), plus the 16-byte wrap boxes of both sets on the
// edge tiles of x-periodic rows.  Four consumer warps pull their 54 values,
// release the stage, run the thermal collision (f: KBC with the Boussinesq
// force; g: relaxation to the Grad equilibrium with the quasi-equilibrium
// of the grid's Prandtl regime), and store their 27 x 32 segments of f and g:
// straight from registers, one 128-byte line per warp and population
// (k_th_tma_d: without an output stage 3 CTAs fit an SM), or through a
// shared-memory stage with one TMA store per set (k_th_tma: 2 CTAs per SM).
// Walls across y or z follow the row rule of the isothermal pass
// (bit j of the tile's bounce mask: source row j lies beyond a wall): f
// bounces back, g takes the anti-bounce-back to the wall equilibrium at rest,
// g_i = -g'_-i + 2 W_i (3 rho T_w + rho~ c_i^2) in deviation form, with the
// density of the node's own state read from global memory.  Tiles with inlet
// or outlet nodes stay on the node-by-node kernel; as in the isothermal pass,
// nodes not updated in the substep are overwritten and rewritten by explode
// and coalesce later in the instant.  Waits are bounded as there.
#include "sc_tma.cuh"
#include "thermal.cuh"

namespace lbmk {

// OUT 0: the output goes through a shared-memory stage and TMA stores (2 CTAs
// per SM fit); OUT 1: each warp stores its rows from registers straight to
// global memory (one 128-byte line per population), and without the output
// stage 3 CTAs per SM fit.
template <typename S, int OUT = 0>
struct ThTmaCfg {
  using C = TmaCfg<S, 2>;
  static constexpr int DI = sizeof(S) == 8 ? 1 : 2;                   // load stages
  static constexpr int HALF = 9 * C::GROUP + 18 * C::SIDE;             // f rows + wrap slots; g follows
  static constexpr int STAGE = 2 * HALF;
  static constexpr int OSTAGE = OUT ? 0 : 2 * 4 * C::OSEGB;           // [set][warp][population][32]
  static constexpr uint32_t TX = 2u * C::TX;
  static constexpr int SMEM = DI * STAGE + OSTAGE + 128;
  static constexpr int THREADS = 160;
  static constexpr int MINB = (OUT && sizeof(S) == 4) ? 3 : 1;        // CTAs per SM the registers aim for
};

template <typename S>
struct ThMaps {
  CUtensorMap f_in, f_out, f_wrap, g_in, g_out, g_wrap;
};

template <typename R, int OUT>
__device__ __forceinline__ void th_tma_body(const ThMaps<R>& m, const PatchDev& p, const R* __restrict__ fin,
                                            R* __restrict__ fout, R* __restrict__ gout,
                                            const unsigned long long* __restrict__ tiles, int ntiles,
                                            const ThParams<R>& tp, int* status) {
  using T = ThTmaCfg<R, OUT>;
  using C = typename T::C;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned char* ostage = smem + T::DI * T::STAGE;
  __shared__ __align__(8) uint64_t full[T::DI], empty[T::DI];
  __shared__ int4 tile_at[T::DI];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nmine = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  if (tid == 0) {
    for (int s = 0; s < T::DI; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 4) {
    // ---------------- producer ----------------
    if (lane != 0) return;
    for (int k = 0; k < nmine; ++k) {
      const int s = k % T::DI;
      if (k >= T::DI && !mbar_wait_bounded(&empty[s], (uint32_t)((k / T::DI) - 1) & 1u)) {
        atomicOr(status, 2);
        return;
      }
      int tx, ty, tz;
      const unsigned long long te = tiles[blockIdx.x + (size_t)k * gridDim.x];
      tile_xyz(te, tx, ty, tz);
      const int bm = tile_bounce(te);
      const bool first = p.span[0] && tx == 0;
      const bool last = p.span[0] && (tx + 1) * C::BX >= p.dim[0];
      tile_at[s] = make_int4(tx, ty, tz, bm);
      const uint32_t txw = 2u * 16u * (uint32_t)(9 - __popc(bm));  // wrap boxes of the rows not bounced
      mbar_expect_tx(&full[s], T::TX + (first ? txw : 0u) + (last ? txw : 0u));
      unsigned char* stage = smem + s * T::STAGE;
      const int x0 = tx * C::BX - C::H;
#pragma unroll 1
      for (int set = 0; set < 2; ++set) {
        unsigned char* half = stage + set * T::HALF;
        unsigned char* side = half + 9 * C::GROUP;
        const CUtensorMap* in = set ? &m.g_in : &m.f_in;
        const CUtensorMap* wr = set ? &m.g_wrap : &m.f_wrap;
#pragma unroll 1
        for (int j = 0; j < 9; ++j) {
          if ((bm >> j) & 1) {
            // beyond a wall: the opposite populations of the tile's own row
            tma_load_row(half + j * C::GROUP, in, &full[s], x0, ty, tz, 3 * (8 - j));
            continue;
          }
          const int sy = wrap_axis(ty - (j % 3 - 1), p.dim[1]);
          const int sz = wrap_axis(tz - (j / 3 - 1), p.dim[2]);
          tma_load_row(half + j * C::GROUP, in, &full[s], x0, sy, sz, 3 * j);
          if (first) tma_load_row(side + j * C::SIDE, wr, &full[s], p.dim[0] - C::H, sy, sz, 3 * j + 2);
          if (last) tma_load_row(side + (9 + j) * C::SIDE, wr, &full[s], 0, sy, sz, 3 * j);
        }
      }
    }
    return;
  }

  // ---------------- consumers (warps 0-3) ----------------
  for (int k = 0; k < nmine; ++k) {
    const int s = k % T::DI;
    if (!mbar_wait_bounded(&full[s], (uint32_t)(k / T::DI) & 1u, tp.wait_sleeps)) {
      // not arrived in time: flag, wait (full bound) for the loads that may
      // still be in flight, this stage's included, drain stores, leave
      if (lane == 0) atomicOr(status, 2);
      for (int j = k; j < nmine && j < k + T::DI; ++j)
        mbar_wait_bounded(&full[j % T::DI], (uint32_t)(j / T::DI) & 1u);
      if (lane == 0) bulk_wait_all();
      return;
    }
    const int4 tc = tile_at[s];
    const int tx = tc.x, y = tc.y, z = tc.z, bm = tc.w;
    const int x = tx * C::BX + tid;
    const R* stf = reinterpret_cast<const R*>(smem + s * T::STAGE);
    const R* stg = reinterpret_cast<const R*>(smem + s * T::STAGE + T::HALF);
    R f[27], g[27];
    if (bm == 0) {
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = stf[row_base<R>(i) + C::H + tid - CX(i)];
        g[i] = stg[row_base<R>(i) + C::H + tid - CX(i)];
      });
    } else {
      // wall rows: density of the node's own post-collision state
      R rho_own_t = 0;
      if (x < p.dim[0]) {
        const long long own = node_index(p, x, y, z);
        unroll<27>([&](auto I) { rho_own_t += fin[(long long)decltype(I)::value * p.plane + own]; });
      }
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int j = i / 3;
        if ((bm >> j) & 1) {
          const int ob = row_base<R>(3 * j + 2 - i % 3) + C::H + tid;
          f[i] = stf[ob];
          // wall face: z wins over y where both lie beyond walls
          const int sy = p.org[1] + y - CY(i), sz = p.org[2] + z - CZ(i);
          int face = -1;
          if (sy < 0) face = 2;
          else if (sy > p.maxc[1]) face = 3;
          if (sz < 0) face = 4;
          else if (sz > p.maxc[2]) face = 5;
          const R tw = face >= 0 ? tp.twd[face] : R(0);
          g[i] = -stg[ob] + R(2 * WI(i)) * (R(3) * (R(1) + rho_own_t) * tw + rho_own_t * R(C2<i>()));
        } else {
          f[i] = stf[row_base<R>(i) + C::H + tid - CX(i)];
          g[i] = stg[row_base<R>(i) + C::H + tid - CX(i)];
        }
      });
    }
    if (p.span[0] && (x == 0 || x == p.dim[0] - 1)) {
      const R* sf = stf + 9 * C::GROUP / (int)sizeof(R);
      const R* sg = stg + 9 * C::GROUP / (int)sizeof(R);
      const bool lo = x == 0;
      unroll<27>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const bool b = (bm >> (i / 3)) & 1;
        if (!b && lo && CX(i) == 1) {
          f[i] = sf[(i / 3) * (C::SIDE / (int)sizeof(R)) + C::H - 1];
          g[i] = sg[(i / 3) * (C::SIDE / (int)sizeof(R)) + C::H - 1];
        }
        if (!b && !lo && CX(i) == -1) {
          f[i] = sf[(9 + i / 3) * (C::SIDE / (int)sizeof(R))];
          g[i] = sg[(9 + i / 3) * (C::SIDE / (int)sizeof(R))];
        }
      });
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (x < p.dim[0]) thermal_collide<R>(f, g, tp.beta, tp.beta1, tp.glam, tp.tref_d, tp.lbgk != 0, tp.pr_gt1 != 0);
    if constexpr (OUT == 1) {
      if (x < p.dim[0]) {
        const long long own = node_index(p, x, y, z);
        unroll<27>([&](auto I) {
          constexpr int i = decltype(I)::value;
          __stcs(fout + (long long)i * p.plane + own, f[i]);
          __stcs(gout + (long long)i * p.plane + own, g[i]);
        });
      }
      continue;
    }
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
    unsigned char* segf = ostage + warp * C::OSEGB;
    unsigned char* segg = ostage + (4 + warp) * C::OSEGB;
    unroll<27>([&](auto I) {
      constexpr int i = decltype(I)::value;
      reinterpret_cast<R*>(segf)[i * C::OSEG + lane] = f[i];
      reinterpret_cast<R*>(segg)[i * C::OSEG + lane] = g[i];
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      tma_store_row(&m.f_out, segf, tx * C::BX + warp * C::OSEG, y, z, 0);
      tma_store_row(&m.g_out, segg, tx * C::BX + warp * C::OSEG, y, z, 0);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
}

// The kernels: through the output stage (registers left to the compiler; 2
// CTAs per SM fit in shared memory) and with direct stores (3 CTAs per SM).
template <typename R>
__global__ void __launch_bounds__(160) k_th_tma(const __grid_constant__ ThMaps<R> m, PatchDev p,
                                                const R* __restrict__ fin, R* __restrict__ fout,
                                                R* __restrict__ gout, const unsigned long long* __restrict__ tiles,
                                                int ntiles, ThParams<R> tp, int* status) {
  th_tma_body<R, 0>(m, p, fin, fout, gout, tiles, ntiles, tp, status);
}

template <typename R>
__global__ void __launch_bounds__(160, ThTmaCfg<R, 1>::MINB) k_th_tma_d(const __grid_constant__ ThMaps<R> m,
                                                                       PatchDev p, const R* __restrict__ fin,
                                                                       R* __restrict__ fout, R* __restrict__ gout,
                                                                       const unsigned long long* __restrict__ tiles,
                                                                       int ntiles, ThParams<R> tp, int* status) {
  th_tma_body<R, 1>(m, p, fin, fout, gout, tiles, ntiles, tp, status);
}

// Nodes of TMA tiles the row rule does not give, recomputed node by node.
template <typename R>
__global__ void __launch_bounds__(128) k_th_nodes(PatchDev p, const R* __restrict__ fin, const R* __restrict__ gin,
                                                  R* __restrict__ fout, R* __restrict__ gout,
                                                  const uint32_t* __restrict__ nodes, long long n, ThParams<R> tp,
                                                  int* status) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const long long own = nodes[k];
  const int x = (int)(own % p.nxp), y = (int)((own / p.nxp) % p.dim[1]);
  const int z = (int)(own / ((long long)p.nxp * p.dim[1]));
  R f[27], g[27];
  pull_th<R>(p, fin, gin, x, y, z, f, g, tp.twd, tp.solid_iso != 0, status);
  thermal_collide<R>(f, g, tp.beta, tp.beta1, tp.glam, tp.tref_d, tp.lbgk != 0, tp.pr_gt1 != 0);
  store2(p, fout, gout, own, f, g);
}

template <typename R, typename T, typename K>
cudaError_t th_tma_go(K kern, int& blocks_per_sm, int& sms) {
  if (blocks_per_sm < 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
    if (e) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, T::THREADS, T::SMEM);
    if (e) return e;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  return cudaSuccess;
}

// 0: k_th_tma_d, direct stores (3 CTAs per SM); 1: k_th_tma, TMA stores through
// the output stage (2 CTAs per SM)
int th_tma_variants() { return 2; }

cudaError_t launch_th_tma(int storage, int variant, const void* const maps[6], const PatchDev& p, const void* fin,
                          void* fout, void* gout, const unsigned long long* tiles, int64_t ntiles,
                          const ThermalLevel& L, int* status, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  if (variant < 0 || variant > 1) return cudaErrorInvalidValue;
  return th_dispatch(storage, [&](auto z) -> cudaError_t {
    using R = decltype(z);
    ThMaps<R> m;
    memcpy(&m.f_in, maps[0], sizeof(CUtensorMap));
    memcpy(&m.f_out, maps[1], sizeof(CUtensorMap));
    memcpy(&m.f_wrap, maps[2], sizeof(CUtensorMap));
    memcpy(&m.g_in, maps[3], sizeof(CUtensorMap));
    memcpy(&m.g_out, maps[4], sizeof(CUtensorMap));
    memcpy(&m.g_wrap, maps[5], sizeof(CUtensorMap));
    auto go = [&](auto kern, auto cfg, int& blocks_per_sm, int& sms) -> cudaError_t {
      using T = decltype(cfg);
      if (cudaError_t e = th_tma_go<R, T>(kern, blocks_per_sm, sms)) return e;
      const int grid = (int)std::min<int64_t>(ntiles, (int64_t)blocks_per_sm * sms);
      kern<<<grid, T::THREADS, T::SMEM, st>>>(m, p, (const R*)fin, (R*)fout, (R*)gout, tiles, (int)ntiles,
                                              th_params<R>(L), status);
      return cudaGetLastError();
    };
    static int bps[2] = {-1, -1}, sms[2] = {0, 0};
    if (variant == 0) return go(k_th_tma_d<R>, ThTmaCfg<R, 1>{}, bps[0], sms[0]);
    return go(k_th_tma<R>, ThTmaCfg<R, 0>{}, bps[1], sms[1]);
  });
}

cudaError_t launch_th_nodes(int storage, const PatchDev& p, const void* fin, const void* gin, void* fout, void* gout,
                            const uint32_t* nodes, int64_t n, const ThermalLevel& L, int* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  return th_dispatch(storage, [&](auto z) {
    using R = decltype(z);
    k_th_nodes<R><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(p, (const R*)fin, (const R*)gin, (R*)fout, (R*)gout,
                                                               nodes, n, th_params<R>(L), status);
    return cudaGetLastError();
  });
}

}  // namespace lbmk
