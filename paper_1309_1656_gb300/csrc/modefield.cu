// qlbm_fourier_field: a real Fourier sum evaluated at every site of a
// periodic box, on the device.  It synthesises the smooth seeded
// perturbations (density, velocity, spin) of the large workloads straight
// into device memory; it holds none of the lattice Boltzmann arithmetic.
//
//   out[s] = offset + scale * sum_m (A_m cos(phi_m(s)) + B_m sin(phi_m(s))),
//   phi_m(s) = 2 pi (kx_m x / nx + ky_m y / ny + kz_m z / nz),
//   s = x + nx (y + ny z).
//
// Evaluation: for a row (y, z) the sum is a trigonometric polynomial in x
// alone.  With psi_m = 2 pi (ky_m y / ny + kz_m z / nz),
//   A cos(theta + psi) + B sin(theta + psi)
//     = cos(theta) (A cos psi + B sin psi) + sin(theta) (B cos psi - A sin psi),
// and cos / sin of theta = 2 pi kx x / nx are even / odd in kx, so each
// block first folds the modes into row coefficients P_j, Q_j (j = |kx|) and
// every site then sums kxmax + 1 terms.  Phases are reduced exactly in
// integers ((k y) mod n) before the one rounding in sincospi.  The row
// coefficients are summed in mode order by one thread each, so the result
// does not depend on the launch.
#include "internal.h"

namespace {

constexpr int kFieldBlock = 256;

struct FourierModes {
    int n;                                   // number of modes
    int kxmax;                               // largest |kx|
    int k[QLBM_FOURIER_MAX_MODES][3];
    double A[QLBM_FOURIER_MAX_MODES], B[QLBM_FOURIER_MAX_MODES];
};

__device__ __forceinline__ int64_t mod_pos(int64_t a, int64_t n)
{
    const int64_t r = a % n;
    return r < 0 ? r + n : r;
}

__global__ void __launch_bounds__(kFieldBlock)
k_fourier_field(const __grid_constant__ FourierModes md, int nx, int ny, int nz, int xblocks, double scale,
                double offset, double *__restrict__ out)
{
    // md arrives by value in the kernel's parameter space (read in place)
    __shared__ double cP[QLBM_FOURIER_MAX_MODES], cQ[QLBM_FOURIER_MAX_MODES];
    __shared__ double P[QLBM_FOURIER_MAX_K + 1], Q[QLBM_FOURIER_MAX_K + 1];
    const int row = blockIdx.x / xblocks;
    const int xb = blockIdx.x - row * xblocks;
    const int y = row % ny, z = row / ny;
    for (int m = threadIdx.x; m < md.n; m += blockDim.x) {
        // psi / pi = 2 ((ky y mod ny) / ny + (kz z mod nz) / nz)
        const double ty = (double)mod_pos((int64_t)md.k[m][1] * y, ny) / (double)ny;
        const double tz = (double)mod_pos((int64_t)md.k[m][2] * z, nz) / (double)nz;
        double sp, cp;
        sincospi(2.0 * (ty + tz), &sp, &cp);
        const double a = md.A[m], b = md.B[m];
        cP[m] = a * cp + b * sp;
        const double q = b * cp - a * sp;
        cQ[m] = md.k[m][0] < 0 ? -q : q;
    }
    __syncthreads();
    if (threadIdx.x <= md.kxmax) {
        const int j = threadIdx.x;
        double p = 0.0, q = 0.0;
        for (int m = 0; m < md.n; ++m) {
            const int kx = md.k[m][0];
            if (kx == j || kx == -j) {
                p += cP[m];
                q += cQ[m];
            }
        }
        P[j] = p;
        Q[j] = q;
    }
    __syncthreads();
    const int x = xb * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double acc = P[0];
    for (int j = 1; j <= md.kxmax; ++j) {
        double s, c;
        sincospi(2.0 * (double)mod_pos((int64_t)j * x, nx) / (double)nx, &s, &c);
        acc += P[j] * c + Q[j] * s;
    }
    out[(int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z)] = offset + scale * acc;
}

}  // namespace

extern "C" int qlbm_fourier_field(const int64_t dims[3], int nmodes, const int32_t *k, const double *A,
                                  const double *B, double scale, double offset, double *out, void *stream)
{
    using qlbm::set_global_error;
    if (!dims || !out || (nmodes > 0 && (!k || !A || !B)))
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_fourier_field: null argument");
    if (nmodes < 0 || nmodes > QLBM_FOURIER_MAX_MODES)
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_fourier_field: nmodes must be in [0, 512]");
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 1 || dims[i] > (1 << 30))
            return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_fourier_field: dims must be in [1, 2^30]");
    const int64_t rows = dims[1] * dims[2];
    const int64_t xblocks = (dims[0] + kFieldBlock - 1) / kFieldBlock;
    if (rows * xblocks > 0x7fffffffLL)
        return set_global_error(QLBM_ERR_INVALID_ARG, "qlbm_fourier_field: box too large for the launch grid");
    static_assert(sizeof(FourierModes) <= 32000, "the modes must fit the kernel parameter space");
    FourierModes md;
    md.n = nmodes;
    md.kxmax = 0;
    for (int m = 0; m < nmodes; ++m) {
        for (int i = 0; i < 3; ++i) {
            if (k[3 * m + i] < -QLBM_FOURIER_MAX_K || k[3 * m + i] > QLBM_FOURIER_MAX_K)
                return set_global_error(QLBM_ERR_INVALID_ARG,
                                        "qlbm_fourier_field: wave-vector components must be in [-64, 64]");
            md.k[m][i] = k[3 * m + i];
        }
        const int ax = md.k[m][0] < 0 ? -md.k[m][0] : md.k[m][0];
        if (ax > md.kxmax) md.kxmax = ax;
        md.A[m] = A[m];
        md.B[m] = B[m];
    }
    // the modes travel as a by-value kernel argument: nothing is allocated
    k_fourier_field<<<(unsigned)(rows * xblocks), kFieldBlock, 0, static_cast<cudaStream_t>(stream)>>>(
        md, (int)dims[0], (int)dims[1], (int)dims[2], (int)xblocks, scale, offset, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_global_error(QLBM_ERR_CUDA, cudaGetErrorString(e));
    return QLBM_OK;
}
