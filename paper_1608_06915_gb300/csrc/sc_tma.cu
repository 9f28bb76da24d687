// Storage dispatch of the TMA stream-collide and the tensor-map encoder.
#include "sc_tma.cuh"

namespace lbmk {

cudaError_t launch_sc_tma(int storage, const TmaLaunchPatch* ps, int n, int variant, int lbgk, int wait_sleeps,
                          int* status, cudaStream_t st) {
  switch (storage) {
    case LBM_FP64:
      return sc_tma_fp64(ps, n, variant, lbgk, wait_sleeps, status, st);
    case LBM_FP32:
      return sc_tma_fp32(ps, n, variant, lbgk, wait_sleeps, status, st);
    case LBM_FP16_SHIFT:
      return sc_tma_fp16(ps, n, variant, lbgk, wait_sleeps, status, st);
    case LBM_BF16_SHIFT:
      return sc_tma_bf16(ps, n, variant, lbgk, wait_sleeps, status, st);
    default:
      return cudaErrorInvalidValue;
  }
}

// scalar kernels 0, 1 for every storage; packed-pair kernels 2, 3 for FP32
// arithmetic (FP32 and 16-bit storage); last, the scalar kernel on 64-node tiles
int sc_tma_variants(int storage) { return storage == LBM_FP64 ? 3 : 5; }

int sc_tma_tile_nodes(int storage, int variant) {
  return variant == sc_tma_variants(storage) - 1 ? 64 : 128;
}

cudaError_t launch_sc_tiles(int storage, const PatchDev& p, const void* fin, void* fout, const uint32_t* tiles,
                            int64_t ntiles, int ntx, double beta, const Force& F, int odd, int lbgk, int* status,
                            cudaStream_t st) {
  switch (storage) {
    case LBM_FP64:
      return sc_tiles_fp64(p, fin, fout, tiles, ntiles, ntx, beta, F, odd, lbgk, status, st);
    case LBM_FP32:
      return sc_tiles_fp32(p, fin, fout, tiles, ntiles, ntx, beta, F, odd, lbgk, status, st);
    case LBM_FP16_SHIFT:
      return sc_tiles_fp16(p, fin, fout, tiles, ntiles, ntx, beta, F, odd, lbgk, status, st);
    case LBM_BF16_SHIFT:
      return sc_tiles_bf16(p, fin, fout, tiles, ntiles, ntx, beta, F, odd, lbgk, status, st);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_sc_nodes(int storage, const PatchDev& p, const void* fin, void* fout, const uint32_t* nodes,
                            int64_t n, double beta, const Force& F, int lbgk, int* status, cudaStream_t st) {
  switch (storage) {
    case LBM_FP64:
      return sc_nodes_fp64(p, fin, fout, nodes, n, beta, F, lbgk, status, st);
    case LBM_FP32:
      return sc_nodes_fp32(p, fin, fout, nodes, n, beta, F, lbgk, status, st);
    case LBM_FP16_SHIFT:
      return sc_nodes_fp16(p, fin, fout, nodes, n, beta, F, lbgk, status, st);
    case LBM_BF16_SHIFT:
      return sc_nodes_bf16(p, fin, fout, nodes, n, beta, F, lbgk, status, st);
    default:
      return cudaErrorInvalidValue;
  }
}

// Tensor map of one population buffer, 4-D [27][nz][ny][nx] with the row
// pitch nxp.  Boxes: loads (W, 1, 1, 3) -- one row of three consecutive
// populations, W of a 128-node tile (kind 0) or of a 64-node tile (kind 3);
// stores (32, 1, 1, 27) -- one warp's segment of all populations; wrap (16
// bytes, 1, 1, 1).  The x extent is the patch's node count, not the
// padded pitch: the padding columns of a ragged row then lie outside the
// tensor, so loads fill them without reading memory and stores skip them.
cudaError_t make_tensor_map(int storage, void* out, const void* base, const PatchDev& p, int kind) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e || !fn) return e ? e : cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  CUtensorMapDataType dt;
  int es, w;
  switch (storage) {
    case LBM_FP64:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64, es = 8, w = TmaCfg<double>::W;
      break;
    case LBM_FP32:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32, es = 4, w = TmaCfg<float>::W;
      break;
    case LBM_FP16_SHIFT:
      dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16, es = 2, w = TmaCfg<__half>::W;
      break;
    case LBM_BF16_SHIFT:
      dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, es = 2, w = TmaCfg<__nv_bfloat16>::W;
      break;
    default:
      return cudaErrorInvalidValue;
  }
  const cuuint64_t dims[4] = {(cuuint64_t)p.dim[0], (cuuint64_t)p.dim[1], (cuuint64_t)p.dim[2], 27};
  const cuuint64_t strides[3] = {(cuuint64_t)p.nxp * es, (cuuint64_t)p.nxp * p.dim[1] * es,
                                 (cuuint64_t)p.plane * es};
  cuuint32_t np = 3;
  if (kind == 1) w = TmaCfg<float>::OSEG, np = 27;  // store box: one warp's 32-node segment
  if (kind == 2) w = 16 / es, np = 1;               // wrap box: 16 bytes
  if (kind == 3) w -= TmaCfg<float>::BX - 64;        // load box of a 64-node tile
  const cuuint32_t box[4] = {(cuuint32_t)w, 1, 1, np};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(out), dt, 4, const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lbmk
