// C ABI of the library (declared in include/qlbm.h): argument checking,
// device memory, AA-parity bookkeeping and error reporting around the
// kernels of kernels.cuh.
#include <stdio.h>
#include <string.h>

#include <string>

#include "internal.h"
#include "fdparams.cuh"
#include "kernels.cuh"

using namespace qlbm;

namespace {

thread_local std::string g_create_err;

int fail(qlbm_ctx *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_err = msg;
    return code;
}

int cuda_fail(qlbm_ctx *h, cudaError_t e, const char *what)
{
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return fail(h, e == cudaErrorMemoryAllocation ? QLBM_ERR_OOM : QLBM_ERR_CUDA, buf);
}

#define CK(h, call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);      \
    } while (0)

size_t field_doubles(const qlbm_ctx *h) { return (size_t)(4 + h->d + 1) * (size_t)h->g.N; }

int ensure_staging(qlbm_ctx *h, size_t bytes)
{
    if (h->staging_bytes >= bytes) return QLBM_OK;
    if (h->staging) cudaFree(h->staging);
    h->staging = nullptr;
    h->staging_bytes = 0;
    CK(h, cudaMalloc(&h->staging, bytes));
    h->staging_bytes = bytes;
    return QLBM_OK;
}

// Reads and clears the device flag word (stream must be idle).
int check_flags(qlbm_ctx *h)
{
    unsigned f = 0;
    CK(h, cudaMemcpyAsync(&f, h->flags, sizeof(f), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (f) {
        CK(h, cudaMemsetAsync(h->flags, 0, sizeof(unsigned), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    // FLAG_FD_UNRESOLVED only reports sites that kept rho' = rho on the
    // Fermi-Dirac path; it is not an error.
    if (f & FLAG_NONFINITE) return fail(h, QLBM_ERR_NONFINITE, "a step met a non-finite moment");
    if (f & FLAG_NONPOSITIVE) return fail(h, QLBM_ERR_NONPOSITIVE_DENSITY, "a step met tr rho <= 0");
    return QLBM_OK;
}

bool valid(qlbm_ctx *h) { return h != nullptr && h->pop != nullptr; }

int64_t site_blocks(const qlbm_ctx *h) { return (int64_t)h->g.nxb * h->g.ny * h->g.nz; }

int ensure_reverse(qlbm_ctx *h)
{
    for (int i = 0; i < 2; ++i)
        if (!h->lam[i]) CK(h, cudaMalloc(&h->lam[i], h->lam_bytes()));
    if (!h->dtau_acc) CK(h, cudaMalloc(&h->dtau_acc, (size_t)site_blocks(h) * sizeof(double)));
    return QLBM_OK;
}

// Steps per replay of the captured step graph (an even number, so a replay
// starts and ends in natural order).
constexpr int kGraphSteps = 32;

// Captures kGraphSteps alternating even/odd step launches once per handle.
// Capture goes through a private stream (the legacy default stream cannot
// be captured); the replay is launched on the handle's stream.
int ensure_graph(qlbm_ctx *h)
{
    if (h->graph) return QLBM_OK;
    cudaStream_t cs = nullptr;
    CK(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = h->stream;
    h->stream = cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int i = 0; e == cudaSuccess && i < kGraphSteps; ++i) e = h->ops->step(h, (i & 1) == 1);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    h->stream = saved;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->graph = nullptr;
        h->use_graph = 0;   // fall back to direct launches of the same kernels
    }
    return QLBM_OK;
}

void free_rollout(qlbm_ctx *h)
{
    if (h->ck) cudaFree(h->ck);
    if (h->seg) cudaFree(h->seg);
    h->ck = h->seg = nullptr;
    h->ck_slots = h->seg_slots = 0;
    h->ro_steps = -1;
}

}  // namespace

namespace qlbm {

// Sum of n doubles in a fixed order (one block), scaled by `scale`.
__global__ void __launch_bounds__(kRedBlock) k_sum_scaled(const double *__restrict__ a, int64_t n, double scale,
                                                          double *__restrict__ out)
{
    double acc[1] = {0.0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc[0] += a[i];
    __shared__ double res[1];
    block_sum_store<1>(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) out[0] = res[0] * scale;
}

}  // namespace qlbm

namespace {

// dJ/dtau = (d omega/d tau) * sum of the per-block accumulators.
int read_dtau(qlbm_ctx *h, double *out)
{
    const double domega_dtau = -h->dt / (h->tau * h->tau);
    k_sum_scaled<<<1, kRedBlock, 0, h->stream>>>(h->dtau_acc, site_blocks(h), domega_dtau, h->red_out);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(out, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return QLBM_OK;
}

int import_lam(qlbm_ctx *h, const double *in, int ptr_kind, void *lam)
{
    const size_t bytes = (size_t)h->b * 4 * (size_t)h->g.N * sizeof(double);
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, bytes);
        if (rc) return rc;
        CK(h, cudaMemcpyAsync(h->staging, in, bytes, cudaMemcpyHostToDevice, h->stream));
        CK(h, h->ops->lam_import(h, h->staging, lam));
    } else {
        CK(h, h->ops->lam_import(h, in, lam));
    }
    return QLBM_OK;
}

int export_lam(qlbm_ctx *h, const void *lam, double *out, int ptr_kind)
{
    const size_t bytes = (size_t)h->b * 4 * (size_t)h->g.N * sizeof(double);
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, bytes);
        if (rc) return rc;
        CK(h, h->ops->lam_export(h, lam, h->staging));
        CK(h, cudaMemcpyAsync(out, h->staging, bytes, cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, h->ops->lam_export(h, lam, out));
    }
    return QLBM_OK;
}

}  // namespace

namespace qlbm {

int set_global_error(int code, const char *msg) { return fail(nullptr, code, msg); }

__global__ void __launch_bounds__(kRedBlock)
k_conserved_final(const double *__restrict__ partials, int nparts, double xi, int64_t N,
                  double *__restrict__ out)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < nparts; r += blockDim.x)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] += partials[(int64_t)r * 8 + i];
    __shared__ double res[8];
    block_sum_store<8>(acc, res);
    __syncthreads();
    if (threadIdx.x < 8) {
        const int i = threadIdx.x;
        const double scale = i < 4 ? 1.0 : (i < 7 ? xi : 0.5 * xi * xi);
        out[i] = res[i] * scale / (double)N;
    }
}

// Unit quaternion of the field term at every site from B [3][N] (double):
// (cos phi, sin phi B/|B|), phi = mu |B| dt, i.e. U(x) = exp(-i mu dt
// sigma.B(x)) (Sec. 5, Eq. sigmaB_comm); the identity where B = 0.
// Non-finite input sets FLAG_NONFINITE.
__device__ __forceinline__ void store_quat(float4 *p, double w, double x, double y, double z)
{
    *p = make_float4((float)w, (float)x, (float)y, (float)z);
}
__device__ __forceinline__ void store_quat(DQuad *p, double w, double x, double y, double z)
{
    p->a = make_double2(w, x);
    p->b = make_double2(y, z);
}

template <class V>
__global__ void __launch_bounds__(256)
k_field_quaternions(const double *__restrict__ B, int64_t N, double mu_dt, V *__restrict__ out,
                    unsigned *__restrict__ flags)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double bx = B[s], by = B[N + s], bz = B[2 * N + s];
    const double nb = sqrt(bx * bx + by * by + bz * bz);
    double w = 1.0, x = 0.0, y = 0.0, z = 0.0;
    if (!(nb < 1e300)) {
        atomicOr(flags, (unsigned)FLAG_NONFINITE);
    } else if (nb > 0.0) {
        double sn, cs;
        sincos(mu_dt * nb, &sn, &cs);
        const double f = sn / nb;
        w = cs;
        x = f * bx;
        y = f * by;
        z = f * bz;
    }
    store_quat(out + s, w, x, y, z);
}

cudaError_t launch_conserved_final(qlbm_ctx *h)
{
    k_conserved_final<<<1, kRedBlock, 0, h->stream>>>(h->partials, h->red_grid ? h->red_grid : h->nred, h->hc.xi,
                                                      h->g.N, h->red_out);
    return cudaGetLastError();
}

}  // namespace qlbm

extern "C" {

int qlbm_create(qlbm_handle *out, int lattice, const int64_t dims[3], double tau, double beta0,
                double dt, int precision, void *stream)
{
    if (!out || !dims) return fail(nullptr, QLBM_ERR_INVALID_ARG, "null argument");
    if (lattice != QLBM_D2Q9 && lattice != QLBM_D3Q19)
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "lattice must be QLBM_D2Q9 or QLBM_D3Q19");
    if (precision != QLBM_FP64 && precision != QLBM_FP32 && precision != QLBM_FP16_DEV && precision != QLBM_DF64 &&
        precision != QLBM_FP64_DF)
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "unknown precision");
    if (!(tau > 0.0) || !(beta0 > 0.0) || !(dt > 0.0))
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "tau, beta0 and dt must be > 0");
    const int d = lattice;
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (d == 2 && dims[2] != 1))
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "dims must be >= 1 (nz = 1 for D2Q9)");
    if (dims[0] > (1 << 30) || dims[1] > (1 << 30) || dims[2] > (1 << 30))
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "dims too large");

    qlbm_ctx *h = new qlbm_ctx();
    h->d = d;
    h->prec = precision;
    h->tau = tau;
    h->beta0 = beta0;
    h->dt = dt;
    h->stream = static_cast<cudaStream_t>(stream);
    compute_constants(d, beta0, &h->hc);
    h->b = h->hc.b;
    h->ops = lattice_ops(d, precision);
    Grid &g = h->g;
    g.nx = (int)dims[0];
    g.ny = (int)dims[1];
    g.nz = (int)dims[2];
    const int bx = (int)site_block(g).x;
    g.nxb = (g.nx + bx - 1) / bx;
    g.N = (int64_t)g.nx * g.ny * g.nz;
    g.P = (g.N + 63) / 64 * 64;
    if ((int64_t)g.nxb * g.ny * g.nz > 0x7fffffffLL) {
        delete h;
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "lattice too large for the launch grid");
    }
    if (g.P > 0x7fffffffLL) {   // the kernels index sites with 32-bit integers
        delete h;
        return fail(nullptr, QLBM_ERR_INVALID_ARG, "lattice too large: at most 2^31 - 64 sites");
    }
    h->elem_bytes =
        (precision == QLBM_FP64 || precision == QLBM_DF64 || precision == QLBM_FP64_DF) ? 8 : (precision == QLBM_FP32 ? 4 : 2);

    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    size_t bytes = (size_t)h->b * 4 * (size_t)g.P * h->elem_bytes;
    if (e == cudaSuccess) e = cudaMalloc(&h->pop, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->flags, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    int64_t nred = (g.N + kRedBlock - 1) / kRedBlock;
    h->nred = (int)(nred < 1024 ? nred : 1024);
    if (e == cudaSuccess) e = cudaMalloc(&h->partials, (size_t)h->nred * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->red_out, 8 * sizeof(double));
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "qlbm_create: %s (population buffer %zu bytes)",
                 cudaGetErrorString(e), bytes);
        qlbm_destroy(h);
        cudaGetLastError();
        return fail(nullptr, e == cudaErrorMemoryAllocation ? QLBM_ERR_OOM : QLBM_ERR_CUDA, buf);
    }
    *out = h;
    return QLBM_OK;
}

void qlbm_destroy(qlbm_handle h)
{
    if (!h) return;
    if (h->stream || h->pop) cudaStreamSynchronize(h->stream);
    if (h->pop) cudaFree(h->pop);
    if (h->flags) cudaFree(h->flags);
    if (h->partials) cudaFree(h->partials);
    if (h->red_out) cudaFree(h->red_out);
    if (h->staging) cudaFree(h->staging);
    for (int i = 0; i < 2; ++i)
        if (h->lam[i]) cudaFree(h->lam[i]);
    if (h->dtau_acc) cudaFree(h->dtau_acc);
    if (h->scratch_state) cudaFree(h->scratch_state);
    if (h->fd_fail) cudaFree(h->fd_fail);
    if (h->qfield) cudaFree(h->qfield);
    if (h->neg_count) cudaFree(h->neg_count);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    free_rollout(h);
    delete h;
}

const char *qlbm_last_error(qlbm_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int qlbm_info(qlbm_handle h, double *out, int n)
{
    if (!valid(h) || !out || n < 16) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_info: bad argument");
    const HostConsts &k = h->hc;
    const double v[16] = {(double)k.d, (double)k.b, k.xi,     k.a,      k.w[0], k.w[1],
                          k.w[2],      k.c,         k.m,      k.alpha3, k.alpha4, k.alpha5,
                          h->tau,      h->beta0,    h->dt,    (double)h->prec};
    memcpy(out, v, sizeof(v));
    return QLBM_OK;
}

int qlbm_init_equilibrium(qlbm_handle h, const double *rho4, const double *u, const double *eps,
                          int ptr_kind)
{
    if (!valid(h) || !rho4 || !u) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_init_equilibrium: null argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE)
        return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    const size_t N = (size_t)h->g.N;
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, field_doubles(h) * sizeof(double));
        if (rc) return rc;
        double *r = h->staging, *uu = r + 4 * N, *ee = uu + (size_t)h->d * N;
        CK(h, cudaMemcpyAsync(r, rho4, 4 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(uu, u, (size_t)h->d * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        if (eps) CK(h, cudaMemcpyAsync(ee, eps, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, h->ops->init_eq(h, r, uu, eps ? ee : nullptr));
        CK(h, cudaStreamSynchronize(h->stream));
    } else {
        CK(h, h->ops->init_eq(h, rho4, u, eps));
    }
    h->parity = 0;
    h->t = 0;
    h->ro_steps = -1;
    return QLBM_OK;
}

int qlbm_step(qlbm_handle h, int64_t nsteps)
{
    if (!valid(h) || nsteps < 0) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_step: bad argument");
    if (nsteps > 0) h->ro_steps = -1;   // a recorded rollout no longer ends at the current state
    if (h->eq_path == QLBM_EQ_FD_PARAMS) {
        for (int64_t i = 0; i < nsteps; ++i) {
            CK(h, h->ops->step_fd(h, h->parity == 1));
            h->parity ^= 1;
            h->t += 1;
        }
        return QLBM_OK;
    }
    if (h->use_graph && nsteps >= 2 * kGraphSteps) {
        if (h->parity == 1) {   // bring the buffer to natural order first
            CK(h, h->ops->step(h, true));
            h->parity = 0;
            h->t += 1;
            --nsteps;
        }
        int rc = ensure_graph(h);
        if (rc) return rc;
        while (h->graph && nsteps >= kGraphSteps) {
            CK(h, cudaGraphLaunch(h->graph, h->stream));
            h->t += kGraphSteps;
            nsteps -= kGraphSteps;
        }
    }
    for (int64_t i = 0; i < nsteps; ++i) {
        const bool odd = h->parity == 1;
        CK(h, h->ops->step(h, odd));
        h->parity ^= 1;
        h->t += 1;
    }
    return QLBM_OK;
}

int64_t qlbm_time(qlbm_handle h) { return h ? h->t : -1; }

int qlbm_sync(qlbm_handle h)
{
    if (!valid(h)) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_sync: bad handle");
    CK(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

int qlbm_moments(qlbm_handle h, double *rho4, double *u, double *eps, int ptr_kind)
{
    if (!valid(h)) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_moments: bad handle");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE)
        return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    const size_t N = (size_t)h->g.N;
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, field_doubles(h) * sizeof(double));
        if (rc) return rc;
        double *r = h->staging, *uu = r + 4 * N, *ee = uu + (size_t)h->d * N;
        CK(h, h->ops->moments(h, rho4 ? r : nullptr, u ? uu : nullptr, eps ? ee : nullptr));
        if (rho4) CK(h, cudaMemcpyAsync(rho4, r, 4 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (u) CK(h, cudaMemcpyAsync(u, uu, (size_t)h->d * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (eps) CK(h, cudaMemcpyAsync(eps, ee, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, h->ops->moments(h, rho4, u, eps));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

int qlbm_conserved(qlbm_handle h, double *out)
{
    if (!valid(h) || !out) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_conserved: bad argument");
    CK(h, h->ops->conserved_partial(h));
    CK(h, launch_conserved_final(h));
    CK(h, cudaMemcpyAsync(out, h->red_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

int qlbm_get_state(qlbm_handle h, double *buf, int ptr_kind)
{
    if (!valid(h) || !buf) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_get_state: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE)
        return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    const size_t bytes = (size_t)h->b * 4 * (size_t)h->g.N * sizeof(double);
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, bytes);
        if (rc) return rc;
        CK(h, h->ops->get_state(h, h->staging));
        CK(h, cudaMemcpyAsync(buf, h->staging, bytes, cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, h->ops->get_state(h, buf));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

int qlbm_set_state(qlbm_handle h, const double *buf, int ptr_kind)
{
    if (!valid(h) || !buf) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_state: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE)
        return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    const size_t bytes = (size_t)h->b * 4 * (size_t)h->g.N * sizeof(double);
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, bytes);
        if (rc) return rc;
        CK(h, cudaMemcpyAsync(h->staging, buf, bytes, cudaMemcpyHostToDevice, h->stream));
        CK(h, h->ops->set_state(h, h->staging));
        CK(h, cudaStreamSynchronize(h->stream));
    } else {
        CK(h, h->ops->set_state(h, buf));
    }
    h->parity = 0;
    h->t = 0;
    h->ro_steps = -1;
    return QLBM_OK;
}

// A checkpoint image is compact: the natural-order planes without their
// padding (b planes of N vectors; double-float storage 2b planes).
namespace {
int64_t image_planes(const qlbm_ctx *h) { return (int64_t)h->b * (h->prec == QLBM_DF64 ? 2 : 1); }
size_t vector_bytes(const qlbm_ctx *h) { return 4 * h->elem_bytes / (h->prec == QLBM_DF64 ? 2 : 1); }
}  // namespace

int64_t qlbm_checkpoint_bytes(qlbm_handle h)
{
    return valid(h) ? image_planes(h) * h->g.N * (int64_t)vector_bytes(h) : -1;
}

int qlbm_save_checkpoint(qlbm_handle h, void *buf, int ptr_kind)
{
    if (!valid(h) || !buf) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_save_checkpoint: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    int rc = ensure_staging(h, h->state_bytes());
    if (rc) return rc;
    CK(h, h->ops->copy_natural(h, h->staging));
    const size_t row = (size_t)h->g.N * vector_bytes(h), pitch = (size_t)h->g.P * vector_bytes(h);
    const cudaMemcpyKind kind = ptr_kind == QLBM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    for (int64_t p = 0; p < image_planes(h); ++p)
        CK(h, cudaMemcpyAsync(static_cast<char *>(buf) + p * row, reinterpret_cast<char *>(h->staging) + p * pitch,
                              row, kind, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

int qlbm_load_checkpoint(qlbm_handle h, const void *buf, int ptr_kind)
{
    if (!valid(h) || !buf) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_load_checkpoint: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    const size_t row = (size_t)h->g.N * vector_bytes(h), pitch = (size_t)h->g.P * vector_bytes(h);
    const cudaMemcpyKind kind = ptr_kind == QLBM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int64_t p = 0; p < image_planes(h); ++p)
        CK(h, cudaMemcpyAsync(static_cast<char *>(h->pop) + p * pitch, static_cast<const char *>(buf) + p * row, row,
                              kind, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->parity = 0;
    h->t = 0;
    h->ro_steps = -1;
    return QLBM_OK;
}

int qlbm_step_adjoint(qlbm_handle h, const double *lam_next, double *lam, double *dJ_dtau, int ptr_kind)
{
    if (!valid(h) || !lam_next || !lam) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_step_adjoint: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (!h->ops->adjoint) return fail(h, QLBM_ERR_UNSUPPORTED, "qlbm_step_adjoint: no reverse mode for this precision");
    int rc = ensure_reverse(h);
    if (rc) return rc;
    const void *state = h->pop;
    if (h->parity) {
        if (!h->scratch_state) CK(h, cudaMalloc(&h->scratch_state, h->state_bytes()));
        CK(h, h->ops->copy_natural(h, h->scratch_state));
        state = h->scratch_state;
    }
    if ((rc = import_lam(h, lam_next, ptr_kind, h->lam[0]))) return rc;
    CK(h, cudaMemsetAsync(h->dtau_acc, 0, (size_t)site_blocks(h) * sizeof(double), h->stream));
    CK(h, h->ops->adjoint(h, state, h->lam[0], h->lam[1]));
    if ((rc = export_lam(h, h->lam[1], lam, ptr_kind))) return rc;
    double g = 0.0;
    if ((rc = read_dtau(h, &g))) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    if (dJ_dtau) *dJ_dtau = g;
    return check_flags(h);
}

int qlbm_rollout(qlbm_handle h, int64_t nsteps, int64_t interval)
{
    if (!valid(h) || nsteps < 0 || interval < 0) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_rollout: bad argument");
    if (h->eq_path != QLBM_EQ_DIRECT)
        return fail(h, QLBM_ERR_UNSUPPORTED, "qlbm_rollout: the reverse mode covers the direct equilibrium path");
    if (!h->ops->adjoint) return fail(h, QLBM_ERR_UNSUPPORTED, "qlbm_rollout: no reverse mode for this precision");
    const size_t sb = h->state_bytes();
    int64_t K = interval;
    if (K == 0) {
        // automatic: keep every state when they fit in 3/4 of the device
        // memory available to the handle (no recomputation in the reverse
        // sweep), else square-root checkpointing
        size_t free_b = 0, total_b = 0;
        CK(h, cudaMemGetInfo(&free_b, &total_b));
        const double avail = (double)free_b + (double)(h->ck_slots + h->seg_slots) * (double)sb;
        if ((double)nsteps * (double)sb <= 0.75 * avail) {
            K = 1;
        } else {
            K = 1;
            while (K * K < nsteps) ++K;
        }
    }
    int64_t nseg = (nsteps + K - 1) / K;
    int64_t need_seg = K > 1 ? K - 1 : 0;
    if (h->ck_slots < nseg || h->seg_slots < need_seg) {
        free_rollout(h);
        if (nseg > 0) {
            cudaError_t e = cudaMalloc(&h->ck, sb * (size_t)nseg);
            if (e == cudaSuccess && need_seg > 0) e = cudaMalloc(&h->seg, sb * (size_t)need_seg);
            if (e != cudaSuccess && interval == 0 && K == 1 && nsteps > 1) {
                // the automatic choice did not fit after all: square-root checkpoints
                cudaGetLastError();
                free_rollout(h);
                K = 1;
                while (K * K < nsteps) ++K;
                nseg = (nsteps + K - 1) / K;
                need_seg = K - 1;
                e = cudaMalloc(&h->ck, sb * (size_t)nseg);
                if (e == cudaSuccess && need_seg > 0) e = cudaMalloc(&h->seg, sb * (size_t)need_seg);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                free_rollout(h);
                char buf[256];
                snprintf(buf, sizeof(buf), "qlbm_rollout: %lld checkpoints + %lld segment states of %zu bytes "
                         "do not fit (%s)", (long long)nseg, (long long)need_seg, sb, cudaGetErrorString(e));
                return fail(h, QLBM_ERR_OOM, buf);
            }
        }
        h->ck_slots = nseg;
        h->seg_slots = need_seg;
    }
    if (K == 1 && nsteps > 0) {
        // every state kept: the two-buffer kernel writes step i's result
        // straight into slot i + 1 (the same bytes as an in-place step), and
        // the last step back into the live buffer in natural order
        char *ck = static_cast<char *>(h->ck);
        CK(h, h->ops->copy_natural(h, ck));
        for (int64_t i = 0; i + 1 < nsteps; ++i) CK(h, h->ops->push(h, ck + sb * (size_t)i, ck + sb * (size_t)(i + 1)));
        CK(h, h->ops->push(h, ck + sb * (size_t)(nsteps - 1), h->pop));
        h->parity = 0;
        h->t += nsteps;
    } else {
        for (int64_t i = 0; i < nsteps; ++i) {
            if (i % K == 0) CK(h, h->ops->copy_natural(h, static_cast<char *>(h->ck) + sb * (size_t)(i / K)));
            CK(h, h->ops->step(h, h->parity == 1));
            h->parity ^= 1;
            h->t += 1;
        }
    }
    h->ro_steps = nsteps;
    h->ro_interval = K;
    h->ro_id += 1;
    return QLBM_OK;
}

int64_t qlbm_rollout_interval(qlbm_handle h) { return (h && h->ro_steps >= 0) ? h->ro_interval : -1; }

int64_t qlbm_rollout_id(qlbm_handle h) { return (h && h->ro_steps >= 0) ? h->ro_id : -1; }

int qlbm_rollout_adjoint(qlbm_handle h, const double *lam_T, double *lam_0, double *dJ_dtau, int ptr_kind)
{
    if (!valid(h) || !lam_T || !lam_0) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_rollout_adjoint: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (!h->ops->adjoint) return fail(h, QLBM_ERR_UNSUPPORTED, "qlbm_rollout_adjoint: no reverse mode for this precision");
    if (h->ro_steps < 0) return fail(h, QLBM_ERR_STATE, "qlbm_rollout_adjoint: no rollout recorded");
    int rc = ensure_reverse(h);
    if (rc) return rc;
    if ((rc = import_lam(h, lam_T, ptr_kind, h->lam[0]))) return rc;
    CK(h, cudaMemsetAsync(h->dtau_acc, 0, (size_t)site_blocks(h) * sizeof(double), h->stream));
    const int64_t N = h->ro_steps, K = h->ro_interval;
    const size_t sb = h->state_bytes();
    int cur = 0;
    for (int64_t seg = (N + K - 1) / K - 1; seg >= 0; --seg) {
        const int64_t len = (N - seg * K) < K ? (N - seg * K) : K;
        auto slot = [&](int64_t j) -> void * {
            return j == 0 ? static_cast<char *>(h->ck) + sb * (size_t)seg
                          : static_cast<char *>(h->seg) + sb * (size_t)(j - 1);
        };
        for (int64_t j = 1; j < len; ++j) CK(h, h->ops->push(h, slot(j - 1), slot(j)));
        for (int64_t j = len - 1; j >= 0; --j) {
            CK(h, h->ops->adjoint(h, slot(j), h->lam[cur], h->lam[1 - cur]));
            cur ^= 1;
        }
    }
    if ((rc = export_lam(h, h->lam[cur], lam_0, ptr_kind))) return rc;
    double g = 0.0;
    if ((rc = read_dtau(h, &g))) return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    if (dJ_dtau) *dJ_dtau = g;
    return check_flags(h);
}

int qlbm_init_equilibrium_adjoint(qlbm_handle h, const double *rho4, const double *u, const double *eps,
                                  const double *lam0, double *g_rho4, double *g_u, double *g_eps, int ptr_kind)
{
    if (!valid(h) || !rho4 || !u || !lam0)
        return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_init_equilibrium_adjoint: null argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (ptr_kind == QLBM_DEVICE) {
        CK(h, h->ops->init_adjoint(h, lam0, rho4, u, eps, g_rho4, g_u, g_eps));
        CK(h, cudaStreamSynchronize(h->stream));
        return QLBM_OK;
    }
    const size_t N = (size_t)h->g.N, fd = field_doubles(h), ld = (size_t)h->b * 4 * N;
    int rc = ensure_staging(h, (2 * fd + ld) * sizeof(double));
    if (rc) return rc;
    double *r = h->staging, *uu = r + 4 * N, *ee = uu + (size_t)h->d * N;
    double *gr = h->staging + fd, *gu = gr + 4 * N, *ge = gu + (size_t)h->d * N;
    double *l = h->staging + 2 * fd;
    CK(h, cudaMemcpyAsync(r, rho4, 4 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(uu, u, (size_t)h->d * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (eps) CK(h, cudaMemcpyAsync(ee, eps, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(l, lam0, ld * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, h->ops->init_adjoint(h, l, r, uu, eps ? ee : nullptr, gr, gu, ge));
    if (g_rho4) CK(h, cudaMemcpyAsync(g_rho4, gr, 4 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (g_u) CK(h, cudaMemcpyAsync(g_u, gu, (size_t)h->d * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (g_eps) CK(h, cudaMemcpyAsync(g_eps, ge, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return QLBM_OK;
}

int qlbm_init_fd_params(qlbm_handle h, const double *beta, const double *mu_up, const double *mu_dn,
                        const double *axis, const double *u, int ptr_kind)
{
    if (!valid(h) || !beta || !mu_up || !mu_dn || !axis || !u)
        return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_init_fd_params: null argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    const size_t N = (size_t)h->g.N;
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, (6 + (size_t)h->d) * N * sizeof(double));
        if (rc) return rc;
        double *b = h->staging, *mu = b + N, *md = mu + N, *ax = md + N, *uu = ax + 3 * N;
        CK(h, cudaMemcpyAsync(b, beta, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(mu, mu_up, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(md, mu_dn, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(ax, axis, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(uu, u, (size_t)h->d * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(h, h->ops->init_fd(h, b, mu, md, ax, uu));
        CK(h, cudaStreamSynchronize(h->stream));
    } else {
        CK(h, h->ops->init_fd(h, beta, mu_up, mu_dn, axis, u));
    }
    h->parity = 0;
    h->t = 0;
    h->ro_steps = -1;
    return QLBM_OK;
}

int qlbm_set_magnetic_field(qlbm_handle h, double mu, const double B[3])
{
    if (!valid(h) || !B) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_magnetic_field: bad argument");
    const double nb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    if (!(nb == nb) || !(mu == mu)) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_magnetic_field: NaN");
    double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    int mag = 0;
    if (nb > 0.0 && mu != 0.0) {
        // rotation by theta = 2 mu |B| dt about B/|B| (Rodrigues)
        const double th = 2.0 * mu * nb * h->dt, c = cos(th), s = sin(th), C = 1.0 - c;
        const double x = B[0] / nb, y = B[1] / nb, z = B[2] / nb;
        const double r[9] = {c + x * x * C,     x * y * C - z * s, x * z * C + y * s,
                             y * x * C + z * s, c + y * y * C,     y * z * C - x * s,
                             z * x * C - y * s, z * y * C + x * s, c + z * z * C};
        for (int i = 0; i < 9; ++i) rot[i] = r[i];
        mag = 1;
    }
    for (int i = 0; i < 9; ++i) h->rot[i] = rot[i];
    h->mag = mag;
    if (h->graph) {   // the captured launches carry the old field
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->ro_steps = -1;
    return QLBM_OK;
}

int qlbm_set_magnetic_field_array(qlbm_handle h, double mu, const double *B, int ptr_kind)
{
    if (!valid(h) || !B) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_magnetic_field_array: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (!(mu == mu) || !(fabs(mu) < 1e300))
        return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_magnetic_field_array: mu must be finite");
    const int64_t N = h->g.N;
    // quaternions as doubles for the 64-bit precisions (the double-float
    // steps split them), as floats for the single-precision arithmetic
    const bool dbl = h->prec == QLBM_FP64 || h->prec == QLBM_FP64_DF || h->prec == QLBM_DF64;
    const size_t vb = dbl ? sizeof(DQuad) : sizeof(float4);
    if (!h->qfield) CK(h, cudaMalloc(&h->qfield, (size_t)N * vb));
    const double *src = B;
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, 3 * (size_t)N * sizeof(double));
        if (rc) return rc;
        CK(h, cudaMemcpyAsync(h->staging, B, 3 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        src = h->staging;
    }
    // earlier steps' flags are reported first, so that a bad field is not
    // mistaken for them
    CK(h, cudaStreamSynchronize(h->stream));
    int rc = check_flags(h);
    if (rc) return rc;
    const unsigned nb = (unsigned)((N + 255) / 256);
    if (dbl)
        k_field_quaternions<<<nb, 256, 0, h->stream>>>(src, N, mu * h->dt, static_cast<DQuad *>(h->qfield), h->flags);
    else
        k_field_quaternions<<<nb, 256, 0, h->stream>>>(src, N, mu * h->dt, static_cast<float4 *>(h->qfield), h->flags);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(h->stream));
    if (check_flags(h) != QLBM_OK) {
        h->mag = FIELD_NONE;
        return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_magnetic_field_array: non-finite field value (field switched off)");
    }
    h->mag = FIELD_SITE;
    if (h->graph) {   // the captured launches carry the previous field variant
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->ro_steps = -1;
    return QLBM_OK;
}

int qlbm_set_equilibrium_path(qlbm_handle h, int path)
{
    if (!valid(h)) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_equilibrium_path: bad handle");
    if (path != QLBM_EQ_DIRECT && path != QLBM_EQ_FD_PARAMS)
        return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_set_equilibrium_path: unknown path");
    if (path == QLBM_EQ_FD_PARAMS && !h->ops->step_fd)
        return fail(h, QLBM_ERR_UNSUPPORTED, "the Fermi-Dirac equilibrium path needs FP64 storage (QLBM_FP64 or QLBM_FP64_DF)");
    h->eq_path = path;
    h->ro_steps = -1;
    return QLBM_OK;
}

int qlbm_fd_params(qlbm_handle h, double *beta, double *mu_up, double *mu_dn, double *axis, int64_t *nfail,
                   int ptr_kind)
{
    if (!valid(h)) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_fd_params: bad handle");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (!h->fd_fail) CK(h, cudaMalloc(&h->fd_fail, sizeof(unsigned long long)));
    CK(h, cudaMemsetAsync(h->fd_fail, 0, sizeof(unsigned long long), h->stream));
    const size_t N = (size_t)h->g.N;
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, 6 * N * sizeof(double));
        if (rc) return rc;
        double *b = h->staging, *mu = b + N, *md = mu + N, *ax = md + N;
        CK(h, h->ops->fd_params(h, beta ? b : nullptr, mu_up ? mu : nullptr, mu_dn ? md : nullptr,
                                axis ? ax : nullptr));
        if (beta) CK(h, cudaMemcpyAsync(beta, b, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (mu_up) CK(h, cudaMemcpyAsync(mu_up, mu, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (mu_dn) CK(h, cudaMemcpyAsync(mu_dn, md, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (axis) CK(h, cudaMemcpyAsync(axis, ax, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    } else {
        CK(h, h->ops->fd_params(h, beta, mu_up, mu_dn, axis));
    }
    unsigned long long nf = 0;
    CK(h, cudaMemcpyAsync(&nf, h->fd_fail, sizeof(nf), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (nfail) *nfail = (int64_t)nf;
    return check_flags(h);
}

int qlbm_step_fd_output(qlbm_handle h, float *beta, float *mu_up, float *mu_dn, float *axis, int64_t *nfail,
                        int ptr_kind)
{
    if (!valid(h) || !beta || !mu_up || !mu_dn || !axis)
        return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_step_fd_output: null argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (!h->ops->step_fdout)
        return fail(h, QLBM_ERR_UNSUPPORTED, "qlbm_step_fd_output: needs QLBM_FP32 or QLBM_FP16_DEV storage");
    if (h->eq_path != QLBM_EQ_DIRECT)
        return fail(h, QLBM_ERR_UNSUPPORTED, "qlbm_step_fd_output: covers the direct equilibrium path");
    if (!h->fd_fail) CK(h, cudaMalloc(&h->fd_fail, sizeof(unsigned long long)));
    const size_t N = (size_t)h->g.N;
    float *b = beta, *mu = mu_up, *md = mu_dn, *ax = axis;
    if (ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, 6 * N * sizeof(float));
        if (rc) return rc;
        b = reinterpret_cast<float *>(h->staging);
        mu = b + N;
        md = mu + N;
        ax = md + N;
    }
    const bool count = nfail != nullptr;
    if (count) CK(h, cudaMemsetAsync(h->fd_fail, 0, sizeof(unsigned long long), h->stream));
    CK(h, h->ops->step_fdout(h, h->parity == 1, b, mu, md, ax));
    h->parity ^= 1;
    h->t += 1;
    h->ro_steps = -1;
    if (ptr_kind == QLBM_HOST) {
        CK(h, cudaMemcpyAsync(beta, b, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(mu_up, mu, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(mu_dn, md, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(axis, ax, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    }
    if (count || ptr_kind == QLBM_HOST) {
        unsigned long long nf = 0;
        if (count) CK(h, cudaMemcpyAsync(&nf, h->fd_fail, sizeof(nf), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        if (count) *nfail = (int64_t)nf;
        return check_flags(h);
    }
    return QLBM_OK;
}

int qlbm_negative_eq_count(qlbm_handle h, int64_t *count, uint32_t *mask, int ptr_kind)
{
    if (!valid(h) || !count) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_negative_eq_count: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (!h->neg_count) CK(h, cudaMalloc(&h->neg_count, sizeof(unsigned long long)));
    CK(h, cudaMemsetAsync(h->neg_count, 0, sizeof(unsigned long long), h->stream));
    const size_t N = (size_t)h->g.N;
    unsigned *m = reinterpret_cast<unsigned *>(mask);
    if (mask && ptr_kind == QLBM_HOST) {
        int rc = ensure_staging(h, N * sizeof(unsigned));
        if (rc) return rc;
        m = reinterpret_cast<unsigned *>(h->staging);
    }
    CK(h, h->ops->negative_eq(h, h->neg_count, m));
    if (mask && ptr_kind == QLBM_HOST)
        CK(h, cudaMemcpyAsync(mask, m, N * sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    unsigned long long c = 0;
    CK(h, cudaMemcpyAsync(&c, h->neg_count, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *count = (int64_t)c;
    return check_flags(h);
}

int qlbm_fd_params_adjoint(qlbm_handle h, const double *g_beta, const double *g_mu_up, const double *g_mu_dn,
                           const double *g_axis, double *lam, int ptr_kind)
{
    if (!valid(h) || !lam) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_fd_params_adjoint: bad argument");
    if (ptr_kind != QLBM_HOST && ptr_kind != QLBM_DEVICE) return fail(h, QLBM_ERR_INVALID_ARG, "bad ptr_kind");
    if (ptr_kind == QLBM_DEVICE) {
        CK(h, h->ops->fd_params_adjoint(h, g_beta, g_mu_up, g_mu_dn, g_axis, lam));
        CK(h, cudaStreamSynchronize(h->stream));
        return check_flags(h);
    }
    const size_t N = (size_t)h->g.N, ld = (size_t)h->b * 4 * N;
    int rc = ensure_staging(h, (6 * N + ld) * sizeof(double));
    if (rc) return rc;
    double *gb = h->staging, *gu = gb + N, *gd = gu + N, *ga = gd + N, *l = ga + 3 * N;
    if (g_beta) CK(h, cudaMemcpyAsync(gb, g_beta, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (g_mu_up) CK(h, cudaMemcpyAsync(gu, g_mu_up, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (g_mu_dn) CK(h, cudaMemcpyAsync(gd, g_mu_dn, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (g_axis) CK(h, cudaMemcpyAsync(ga, g_axis, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, h->ops->fd_params_adjoint(h, g_beta ? gb : nullptr, g_mu_up ? gu : nullptr, g_mu_dn ? gd : nullptr,
                                    g_axis ? ga : nullptr, l));
    CK(h, cudaMemcpyAsync(lam, l, ld * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

}  // extern "C"
