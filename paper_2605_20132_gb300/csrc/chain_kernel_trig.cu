// The single-stream chain kernel with the trigger summaries fused into its
// detector (filark_chain_push_triggers): the same kernel as chain_kernel.cu
// instantiated with TRIG, in a translation unit of its own so that the two
// sets build in parallel.
#include "chain_body.cuh"

namespace filark {

namespace {

template <int NS, bool DENSE>
__global__ void __launch_bounds__(kThreads, kCTAsPerSM) chain_trig_kernel(const __grid_constant__ ChainParams p) {
    if (p.pdl) pdl_launch_dependents();
    chain_body<NS, true, DENSE, false, true>(p, p.u, p.u.tx0 + (int)blockIdx.x, blockIdx.y);
}

template <int NS, bool DENSE>
cudaError_t configure_trig_t() {
    cudaError_t e = cudaFuncSetAttribute(chain_trig_kernel<NS, DENSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chain_smem_bytes(DENSE));
    if (e == cudaSuccess && kMaxCluster > 8)
        e = cudaFuncSetAttribute(chain_trig_kernel<NS, DENSE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int NS, bool DENSE>
cudaError_t launch_trig_t(const ChainParams &p, int n_tiles, cudaStream_t stream) {
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
    return cudaLaunchKernelEx(&cfg, chain_trig_kernel<NS, DENSE>, p);
}

}  // namespace

cudaError_t configure_chain_trig_kernels() {
    cudaError_t e = configure_trig_t<0, false>();
    if (e == cudaSuccess) e = configure_trig_t<2, false>();
    if (e == cudaSuccess) e = configure_trig_t<2, true>();
    if (e == cudaSuccess) e = configure_trig_t<4, false>();
    if (e == cudaSuccess) e = configure_trig_t<4, true>();
    if (e == cudaSuccess) e = configure_trig_t<8, false>();
    if (e == cudaSuccess) e = configure_trig_t<8, true>();
    return e;
}

cudaError_t launch_chain_trig(const ChainParams &p, int NS, bool dense, int n_tiles, cudaStream_t stream) {
    switch (NS) {
    case 0: return launch_trig_t<0, false>(p, n_tiles, stream);
    case 2: return dense ? launch_trig_t<2, true>(p, n_tiles, stream) : launch_trig_t<2, false>(p, n_tiles, stream);
    case 4: return dense ? launch_trig_t<4, true>(p, n_tiles, stream) : launch_trig_t<4, false>(p, n_tiles, stream);
    case 8: return dense ? launch_trig_t<8, true>(p, n_tiles, stream) : launch_trig_t<8, false>(p, n_tiles, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace filark
