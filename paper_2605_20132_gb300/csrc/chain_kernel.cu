// Single-stream launch of the fused chain kernel (device code in
// chain_body.cuh): one launch per <= 2048 samples of a push (and per tile
// group when the chain runs its tiles in lanes), grid.x = channel tiles from
// u.tx0 on, grid.y = the cluster of time ranges.
#include "chain_body.cuh"

namespace filark {

namespace {

template <int NS, bool DET, bool DENSE>
__global__ void __launch_bounds__(kThreads, kCTAsPerSM) chain_fwd_kernel(const __grid_constant__ ChainParams p) {
    if (p.pdl) pdl_launch_dependents();
    chain_body<NS, DET, DENSE>(p, p.u, p.u.tx0 + (int)blockIdx.x, blockIdx.y);
}

template <int NS, bool DET, bool DENSE>
cudaError_t configure_t() {
    cudaError_t e = cudaFuncSetAttribute(chain_fwd_kernel<NS, DET, DENSE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem_bytes(DENSE));
    if (e == cudaSuccess && kMaxCluster > 8)
        e = cudaFuncSetAttribute(chain_fwd_kernel<NS, DET, DENSE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int NS, bool DET, bool DENSE>
cudaError_t launch_t(const ChainParams &p, int n_tiles, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_tiles, (unsigned)p.u.R, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = chain_smem_bytes(DENSE);
    cfg.stream = stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)p.u.R;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = p.pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, chain_fwd_kernel<NS, DET, DENSE>, p);
}

}  // namespace

size_t chain_smem_bytes(bool dense) {
    return (size_t)(dense ? kSmemFloatsDense : kSmemFloats) * sizeof(float);
}

cudaError_t configure_chain_kernels() {
    cudaError_t e = cudaSuccess;
#define FILARK_CFG(NS, D, X) if (e == cudaSuccess) e = configure_t<NS, D, X>();
    FILARK_CFG(0, false, false) FILARK_CFG(0, true, false)
    FILARK_CFG(2, false, false) FILARK_CFG(2, true, false) FILARK_CFG(2, false, true) FILARK_CFG(2, true, true)
    FILARK_CFG(4, false, false) FILARK_CFG(4, true, false) FILARK_CFG(4, false, true) FILARK_CFG(4, true, true)
    FILARK_CFG(8, false, false) FILARK_CFG(8, true, false) FILARK_CFG(8, false, true) FILARK_CFG(8, true, true)
#undef FILARK_CFG
    if (e == cudaSuccess) e = configure_chain_trig_kernels();
    if (e == cudaSuccess) e = configure_batch_kernels();
    if (e == cudaSuccess) e = configure_batch_kernels_solo();
    return e;
}

cudaError_t launch_chain(const ChainParams &p, int NS, bool det, bool dense, int n_tiles, cudaStream_t stream) {
#define FILARK_L(N) \
    return dense ? (det ? launch_t<N, true, true>(p, n_tiles, stream) : launch_t<N, false, true>(p, n_tiles, stream)) \
                 : (det ? launch_t<N, true, false>(p, n_tiles, stream) : launch_t<N, false, false>(p, n_tiles, stream));
    switch (NS) {
    case 0: return det ? launch_t<0, true, false>(p, n_tiles, stream) : launch_t<0, false, false>(p, n_tiles, stream);
    case 2: FILARK_L(2)
    case 4: FILARK_L(4)
    case 8: FILARK_L(8)
    default: return cudaErrorInvalidValue;
    }
#undef FILARK_L
}

}  // namespace filark
