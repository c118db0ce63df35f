// C ABI of the library (declared in include/qlbm.h): argument checking,
// device memory, AA-parity bookkeeping and error reporting around the
// kernels of kernels.cuh.
#include <stdio.h>
#include <string.h>

#include <string>

#include "internal.h"
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
    if (f & FLAG_NONFINITE) return fail(h, QLBM_ERR_NONFINITE, "a step met a non-finite moment");
    if (f & FLAG_NONPOSITIVE) return fail(h, QLBM_ERR_NONPOSITIVE_DENSITY, "a step met tr rho <= 0");
    return QLBM_OK;
}

bool valid(qlbm_ctx *h) { return h != nullptr && h->pop != nullptr; }

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

cudaError_t launch_conserved_final(qlbm_ctx *h)
{
    k_conserved_final<<<1, kRedBlock, 0, h->stream>>>(h->partials, h->nred, h->hc.xi, h->g.N,
                                                      h->red_out);
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
    if (precision != QLBM_FP64 && precision != QLBM_FP32 && precision != QLBM_FP16_DEV)
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
    h->ops = (d == 2) ? lattice_ops_d2q9(precision) : lattice_ops_d3q19(precision);
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
    h->elem_bytes = precision == QLBM_FP64 ? 8 : (precision == QLBM_FP32 ? 4 : 2);

    cudaError_t e = cudaGetDevice(&h->device);
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
    return QLBM_OK;
}

int qlbm_step(qlbm_handle h, int64_t nsteps)
{
    if (!valid(h) || nsteps < 0) return fail(h, QLBM_ERR_INVALID_ARG, "qlbm_step: bad argument");
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
    return QLBM_OK;
}

}  // extern "C"
