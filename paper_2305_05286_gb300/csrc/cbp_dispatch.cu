// Kernel selection and launch for every decoder variant.
#include "cbp_internal.cuh"

namespace cbp {

static void* select_kernel(const Variant& v) {
  switch (v.alg) {
    case ALG_CBP_SP:
      if (v.fp) return fp_kernel_ptr();
      if (v.lvl) return level_kernel_ptr(v.shrec);
      return v.win ? sp_win_kernel_ptr(v.chk_shared)
                   : sp_kernel_ptr(v.chk_shared, v.fpt, v.wide, v.self_last);
    case ALG_CBP_NMS:
      if (v.lvl) return nms_level_kernel_ptr(v.shrec);
      return minsum_kernel_ptr(v.alg, v.chk_shared, v.rstore);
    case ALG_LBP_NMS:
      if (v.lvl) return lbp_level_kernel_ptr(v.shrec);
      return minsum_kernel_ptr(v.alg, v.chk_shared, v.rstore);
    case ALG_FBP_SP: return v.lvl ? fbp_level_kernel_ptr(v.shrec, v.deg) : flood_kernel_ptr();
  }
  return nullptr;
}

cudaError_t decoder_func_attrs(const Variant& v, cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, select_kernel(v));
}

cudaError_t decoder_set_smem(const Variant& v, int bytes) {
  return cudaFuncSetAttribute(select_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t decoder_occupancy(const Variant& v, int threads, size_t smem, int* ctas) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, select_kernel(v), threads, smem);
}

cudaError_t launch_decoder(const Variant& v, const KParams& p, int grid, int threads,
                           size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<KParams*>(&p)};
  return cudaLaunchKernel(select_kernel(v), dim3(grid), dim3(threads), args, smem, st);
}

cudaError_t launch_multi(bool chk_shared, int fpt, bool self_last, const MultiParams& mp, int grid,
                         int threads, size_t smem, cudaStream_t st) {
  void* args[] = {const_cast<MultiParams*>(&mp)};
  return cudaLaunchKernel(sp_multi_kernel_ptr(chk_shared, fpt, self_last), dim3(grid),
                          dim3(threads), args, smem, st);
}

}  // namespace cbp
