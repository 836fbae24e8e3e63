// Batched persistent launch of the fused chain (device code in chain_body.cuh):
// many independent streams with their own channel counts, chunk lengths and
// carried state, one launch per push of all of them.
//
// Compiled twice: chain_batch.cu (FILARK_BATCH_SOLO 0, clusters of 2, 4 or 8
// CTAs) and chain_batch_solo.cu
// (FILARK_BATCH_SOLO 1, clusters of one CTA with block barriers in the body);
// the two translation units build in parallel and export their entry points
// under FILARK_BATCH_FN(name).
#pragma once

#include "chain_body.cuh"

#if FILARK_BATCH_SOLO
#define FILARK_BATCH_FN(name) name##_solo
#else
#define FILARK_BATCH_FN(name) name
#endif

namespace filark {

namespace {

// Batched chain: a persistent grid of clusters (1, Rb, 1) takes work items
// from a device counter (the host lists them longest push first, so this is
// greedy longest-first scheduling).  An item is a group of channel tiles of one
// stream; its push is a sequence of units of at most Rb x nbc x 32 samples that
// the cluster runs in order, each unit's state written before the next reads
// it (the body's final cluster barrier orders them; the tile's halo columns
// carry their own state, see ChainUnit::halo_in).  A push that needs fewer
// than Rb time ranges shares the cluster among Rb / reff tiles, reff ranks
// each.  CTAs past a unit's time ranges only keep the cluster barriers in
// step.
template <int NS, bool DET, bool DENSE>
__global__ void __launch_bounds__(kThreads, kCTAsPerSM)
    chain_batch_kernel(const __grid_constant__ ChainParams p, const BatchItem *__restrict__ items,
                       int *__restrict__ ctr, const ChainUnit *__restrict__ units) {
    // The item and unit being run live in shared memory: the body reloads
    // their fields where it uses them instead of holding them in registers
    // (the body runs at the 64-register cap), and the loop keeps only j.
    __shared__ int s_item;
    __shared__ BatchItem s_it;
    __shared__ __align__(16) ChainUnit s_unit;
    if (p.pdl) pdl_launch_dependents();
    cg::cluster_group cluster = cg::this_cluster();
    const bool multi = gridDim.y > 1;
    for (;;) {
        if (blockIdx.y == 0 && threadIdx.x == 0) s_item = atomicAdd(&ctr[1], 1);
        if (multi) cluster_sync_release_acquire();
        else __syncthreads();
        const int k = multi ? *cluster.map_shared_rank(&s_item, 0) : s_item;
        if (k >= ctr[0]) {
            // rank 0 keeps its shared memory until every peer has read s_item
            if (multi) cluster_sync_release_acquire();
            break;
        }
        if (threadIdx.x < (int)(sizeof(BatchItem) / 4))
            reinterpret_cast<int *>(&s_it)[threadIdx.x] = __ldg(reinterpret_cast<const int *>(items + k) + threadIdx.x);
        for (int j = 0;; ++j) {
            __syncthreads();   // s_it is written; the previous unit's readers of shared memory are done
            if (j >= s_it.n_units) break;
            {
                const int *src = reinterpret_cast<const int *>(units + s_it.unit0 + j);
                int *dst = reinterpret_cast<int *>(&s_unit);
                for (int q = threadIdx.x; q < (int)(sizeof(ChainUnit) / 4); q += kThreads) dst[q] = __ldg(src + q);
            }
            __syncthreads();
            // tile s_it.tile + sub, time range rr
            const int sub = (int)blockIdx.y / s_it.reff, rr = (int)blockIdx.y - sub * s_it.reff;
            if constexpr (FILARK_BATCH_SOLO) {
                // one CTA per cluster: every CTA runs its unit (reff = R = 1)
                // with block barriers inside the body.  The unit's global
                // writes (state, history ring) reach device scope before the
                // next unit reads them: a block barrier, then one thread's
                // fence, which is cumulative over the writes the barrier
                // ordered before it (the next barrier follows at the loop top).
                chain_body<NS, DET, DENSE, true>(p, s_unit, s_it.tile + sub, rr);
                __syncthreads();
                if (threadIdx.x == 0) __threadfence();
            } else if (sub < s_it.n_tiles && rr < s_unit.R) {
                chain_body<NS, DET, DENSE>(p, s_unit, s_it.tile + sub, rr);
            } else {
#pragma unroll
                for (int q = 0; q < chain_cluster_barriers<NS, DET>(); ++q) cluster_sync_release_acquire();
            }
        }
        // s_item is rewritten next: the body's last cluster barrier already
        // follows every read of it, except when the body has none
        if (chain_cluster_barriers<NS, DET>() == 0) {
            if (multi) cluster_sync_release_acquire();
            else __syncthreads();
        }
    }
}

template <int NS, bool DET, bool DENSE>
cudaError_t configure_batch_t() {
    return cudaFuncSetAttribute(chain_batch_kernel<NS, DET, DENSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)chain_smem_bytes(DENSE));
}

template <int NS, bool DET, bool DENSE>
void batch_config(int cluster, int n_clusters, cudaStream_t stream, bool pdl, cudaLaunchConfig_t &cfg,
                  cudaLaunchAttribute (&attr)[2]) {
    cfg = {};
    cfg.gridDim = dim3((unsigned)n_clusters, (unsigned)cluster, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = chain_smem_bytes(DENSE);
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)cluster;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
}

template <int NS, bool DET, bool DENSE>
cudaError_t launch_batch_t(const ChainParams &p, int cluster, int n_clusters, const BatchItem *items,
                           int *ctr, const ChainUnit *units, cudaStream_t stream) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    batch_config<NS, DET, DENSE>(cluster, n_clusters, stream, p.pdl != 0, cfg, attr);
    return cudaLaunchKernelEx(&cfg, chain_batch_kernel<NS, DET, DENSE>, p, items, ctr, units);
}

template <int NS, bool DET, bool DENSE>
int max_clusters_t(int cluster) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    batch_config<NS, DET, DENSE>(cluster, 1, nullptr, false, cfg, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, chain_batch_kernel<NS, DET, DENSE>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace

cudaError_t FILARK_BATCH_FN(configure_batch_kernels)() {
    cudaError_t e = cudaSuccess;
#define FILARK_CFG(NS, D, X) if (e == cudaSuccess) e = configure_batch_t<NS, D, X>();
    FILARK_CFG(0, false, false) FILARK_CFG(0, true, false)
    FILARK_CFG(2, false, false) FILARK_CFG(2, true, false) FILARK_CFG(2, false, true) FILARK_CFG(2, true, true)
    FILARK_CFG(4, false, false) FILARK_CFG(4, true, false) FILARK_CFG(4, false, true) FILARK_CFG(4, true, true)
    FILARK_CFG(8, false, false) FILARK_CFG(8, true, false) FILARK_CFG(8, false, true) FILARK_CFG(8, true, true)
#undef FILARK_CFG
    return e;
}

#define FILARK_DISPATCH(CALL)                                                                     \
    switch (NS) {                                                                                 \
    case 0: return det ? CALL(0, true, false) : CALL(0, false, false);                            \
    case 2: return dense ? (det ? CALL(2, true, true) : CALL(2, false, true))                     \
                         : (det ? CALL(2, true, false) : CALL(2, false, false));                  \
    case 4: return dense ? (det ? CALL(4, true, true) : CALL(4, false, true))                     \
                         : (det ? CALL(4, true, false) : CALL(4, false, false));                  \
    case 8: return dense ? (det ? CALL(8, true, true) : CALL(8, false, true))                     \
                         : (det ? CALL(8, true, false) : CALL(8, false, false));                  \
    default: break;                                                                               \
    }

cudaError_t FILARK_BATCH_FN(launch_chain_batch)(const ChainParams &p, int NS, bool det, bool dense, int cluster, int n_clusters,
                               const BatchItem *d_items, int *d_ctr, const ChainUnit *d_units,
                               cudaStream_t stream) {
    if (cluster < 1 || cluster > kMaxCluster || n_clusters < 1) return cudaErrorInvalidValue;
#define FILARK_LB(N, D, X) launch_batch_t<N, D, X>(p, cluster, n_clusters, d_items, d_ctr, d_units, stream)
    FILARK_DISPATCH(FILARK_LB)
#undef FILARK_LB
    return cudaErrorInvalidValue;
}

int FILARK_BATCH_FN(batch_max_active_clusters)(int NS, bool det, bool dense, int cluster) {
#define FILARK_MC(N, D, X) max_clusters_t<N, D, X>(cluster)
    FILARK_DISPATCH(FILARK_MC)
#undef FILARK_MC
    return 0;
}

#undef FILARK_DISPATCH

}  // namespace filark
