// tc_gemm_pair.cu -- CTA-pair launches of the tcgen05 product kernel (tc_kernel.cuh) for
// the products of the mixed path: the level products W and X21 at full tile width and the
// Newton-Schulz products R = I - T X and X += X R.  A cluster of two CTAs on two SMs
// computes each 256 x 256 output tile with tcgen05.mma.cta_group::2; each CTA stages its
// own 128 rows of A and half of the B tile.
#include <mutex>

#include "tc_kernel.cuh"

namespace triinv {
namespace tc {

cudaError_t launch_pair(const Ctx &c, int mode, bool trans, bool unit, const Maps &maps, const Terms &terms,
                        const Pipe &pipe, const Tile *d_tiles, const int *d_off, int ctas, const Epi &epi) {
#define TRI_PAIR_CASE(M)                                                                                    \
    case M:                                                                                                 \
        if (trans)                                                                                          \
            return unit ? launch_t<M, true, true, BN, true>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, epi) \
                        : launch_t<M, true, false, BN, true>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, epi); \
        return unit ? launch_t<M, false, true, BN, true>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, epi)    \
                    : launch_t<M, false, false, BN, true>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, epi);
    switch (mode) {
        TRI_PAIR_CASE(MODE_W)
        TRI_PAIR_CASE(MODE_X21)
        TRI_PAIR_CASE(MODE_RES)
        TRI_PAIR_CASE(MODE_UPD)
        default:
            return cudaErrorInvalidValue;
    }
#undef TRI_PAIR_CASE
}

int pair_lists(const Ctx &c) {
    static std::mutex mu;
    static int cached[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    const int dev = c.device >= 0 && c.device < 64 ? c.device : 0;
    if (cached[dev] > 0) return cached[dev];
    int n = 0;
    auto kern = tc_gemm_kernel<MODE_UPD, false, false, BN, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM_BYTES) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (unsigned)c.sm_count);
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = GEMM_SMEM_BYTES;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) n = 0;
    }
    cudaGetLastError();
    // one CTA per SM: at most half the SMs' worth of pairs
    if (n <= 0) n = c.sm_count / 2;
    n = std::max(1, std::min(n, c.sm_count / 2));
    cached[dev] = n;
    return n;
}

}  // namespace tc
}  // namespace triinv
