// qlbm_conserved_static: the global conserved quantities of a caller-owned
// state, computed without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// these sums: code running under another component's memory manager (a
// framework's caching allocator or a fixed, pre-sized arena that owns all of
// the device's memory) and latency-critical loops in which cudaMalloc and
// cudaFree, which may synchronise the whole device, are not acceptable.  For
// them this entry point takes the state and the output as caller-provided
// device buffers and keeps its only scratch, the per-block partial sums, in
// one file-scope __device__ array of fixed size that lives in the library's
// module on every GPU that loads it, until the process exits.
#include <mutex>

#include "internal.h"
#include "kernels.cuh"

namespace {

// One row of 8 partial sums per block; the reduction never launches more
// than kStaticBlocks blocks (it loops over the sites), so 64 KiB suffice for
// any lattice size.
constexpr int kStaticBlocks = QLBM_STATIC_SCRATCH_BLOCKS;
static __device__ __align__(256) double g_static_partials[kStaticBlocks * 8];

// Device address of g_static_partials per device ordinal.  In host code the
// array's name only stands in for the symbol, so its address on the current
// device is looked up once, with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_partials_addr[kMaxDevices] = {};

int static_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return qlbm::set_global_error(QLBM_ERR_CUDA, "qlbm_conserved_static: cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices)
        return qlbm::set_global_error(QLBM_ERR_UNSUPPORTED, "qlbm_conserved_static: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return qlbm::set_global_error(QLBM_ERR_CUDA,
                                          "qlbm_conserved_static: cudaGetSymbolAddress of the scratch failed");
        }
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *out = g_partials_addr[dev];
    return QLBM_OK;
}

// Partial sums of Eqs. GlobalDensity, GlobalVelocity, GlobalTotalEnergy over
// a canonical state double [b][4][N] (grid-stride; row blockIdx.x of
// partials).  Same sums as k_conserved_partial, read from the canonical
// layout instead of the AA-ordered population buffer.
template <int D>
__global__ void __launch_bounds__(qlbm::kRedBlock)
k_conserved_partial_canonical(const double *__restrict__ state, int64_t N, double *__restrict__ partials)
{
    using namespace qlbm;
    constexpr int Q = Lattice<D>::Q;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += stride) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double *p = state + (int64_t)(4 * q) * N + s;
            const double fq = p[0];
            acc[0] += fq;
            acc[1] += p[N];
            acc[2] += p[2 * N];
            acc[3] += p[3 * N];
            acc[4] += cx<D>(q) * fq;
            acc[5] += cy<D>(q) * fq;
            acc[6] += cz<D>(q) * fq;
            acc[7] += cnorm2<D>(q) * fq;
        }
    }
    block_sum_store<8>(acc, partials + (int64_t)blockIdx.x * 8);
}

}  // namespace

extern "C" int qlbm_conserved_static(int lattice, const int64_t dims[3], double beta0,
                                     const double *state, double *out, void *stream)
{
    using namespace qlbm;
    if (!dims || !state || !out)
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_conserved_static: null argument");
    if (lattice != QLBM_D2Q9 && lattice != QLBM_D3Q19)
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_conserved_static: lattice must be QLBM_D2Q9 or QLBM_D3Q19");
    if (!(beta0 > 0.0))
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_conserved_static: beta0 must be > 0");
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (lattice == QLBM_D2Q9 && dims[2] != 1))
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_conserved_static: dims must be >= 1 (nz = 1 for D2Q9)");
    if (dims[0] > QLBM_STATIC_MAX_SITES || dims[1] > QLBM_STATIC_MAX_SITES ||
        dims[2] > QLBM_STATIC_MAX_SITES ||
        dims[0] * dims[1] > QLBM_STATIC_MAX_SITES || dims[0] * dims[1] * dims[2] > QLBM_STATIC_MAX_SITES)
        return set_global_error(QLBM_ERR_INVALID_ARG,
                                "qlbm_conserved_static: more than QLBM_STATIC_MAX_SITES sites");
    const int64_t N = dims[0] * dims[1] * dims[2];
    HostConsts hc;
    compute_constants(lattice, beta0, &hc);
    double *partials = nullptr;
    int rc = static_scratch(&partials);
    if (rc != QLBM_OK) return rc;
    const int64_t want = (N + kRedBlock - 1) / kRedBlock;
    const int nblocks = (int)(want < kStaticBlocks ? want : kStaticBlocks);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Every row 0..nblocks-1 is written by the first kernel before the second
    // reads it, so nothing left by an earlier call needs clearing.
    if (lattice == QLBM_D2Q9)
        k_conserved_partial_canonical<2><<<nblocks, kRedBlock, 0, st>>>(state, N, partials);
    else
        k_conserved_partial_canonical<3><<<nblocks, kRedBlock, 0, st>>>(state, N, partials);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_conserved_final<<<1, kRedBlock, 0, st>>>(partials, nblocks, hc.xi, N, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_global_error(QLBM_ERR_CUDA, "qlbm_conserved_static: kernel launch failed");
    return QLBM_OK;
}
