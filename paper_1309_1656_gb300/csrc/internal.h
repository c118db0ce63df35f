// Host-side context of a lattice and the per-lattice kernel dispatch table.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/qlbm.h"
#include "lattice.cuh"

namespace qlbm {

// Lattice constants in double, derived on the host from the quadrature's and
// the equilibrium's moment conditions (see consts.cu).
struct HostConsts {
    int d, b;
    double beta0;
    double c, m;          // beta0 <w>_0 and beta0^2 <w^2>_0, w = |p|^2/2
    double xi, a;
    double w[3];          // weights by |i|^2 = 0, 1, 2
    double alpha3, alpha4, alpha5;
    double K;             // beta0 xi^2 / 2
    double eps0;          // c / beta0
};

int compute_constants(int d, double beta0, HostConsts *out);

struct LatticeOps;

}  // namespace qlbm

struct qlbm_ctx {
    int d = 0, b = 0, prec = 0;
    qlbm::Grid g{};
    double tau = 0, beta0 = 0, dt = 0;
    qlbm::HostConsts hc{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 0;                    // streaming multiprocessors of the device
    void *pop = nullptr;            // b*4*P elements of the storage type
    size_t elem_bytes = 0;
    int parity = 0;                 // 1: last written by an even step (swapped)
    int64_t t = 0;                  // steps since init/set_state
    unsigned *flags = nullptr;      // device flag word
    double *partials = nullptr;     // device reduction scratch [nred][8]
    double *red_out = nullptr;      // device [8]
    int nred = 0;                   // rows of partials (the most blocks a reduction launches)
    int red_grid = 0;               // blocks of the reduction: whole waves of resident blocks, <= nred
    double *staging = nullptr;      // device staging for host inputs/outputs
    size_t staging_bytes = 0;
    const qlbm::LatticeOps *ops = nullptr;
    std::string err;
    // reverse mode
    void *lam[2] = {nullptr, nullptr};  // cotangent planes (arithmetic type), natural order
    double *dtau_acc = nullptr;         // per-block dJ/dtau accumulators
    void *scratch_state = nullptr;      // one natural-order state (single adjoint step)
    void *ck = nullptr;                 // rollout checkpoints
    void *seg = nullptr;                // rollout segment states (interval - 1 of them)
    int64_t ck_slots = 0, seg_slots = 0;
    int64_t ro_steps = -1, ro_interval = 0;   // last rollout (-1: none)
    int64_t ro_id = 0;                        // rollouts recorded so far (id of the last one)
    // CUDA graph of kGraphSteps consecutive steps starting from natural order
    cudaGraphExec_t graph = nullptr;
    int use_graph = 1;
    int eq_path = 0;                    // QLBM_EQ_DIRECT or QLBM_EQ_FD_PARAMS
    int mag = 0;                        // magnetic-field term: FIELD_NONE, FIELD_UNIFORM or FIELD_SITE
    void *qfield = nullptr;             // per-site field: N unit quaternions (float4, or DQuad for FP64)
    double rot[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};   // its per-step spin rotation
    unsigned long long *fd_fail = nullptr;   // device counter of unresolved sites
    unsigned long long *neg_count = nullptr; // device counter of the negative-equilibrium diagnostic
    size_t state_bytes() const { return (size_t)b * 4 * (size_t)g.P * elem_bytes; }
    size_t lam_bytes() const { return (size_t)b * 4 * (size_t)g.P * (prec == QLBM_FP64 ? 8 : 4); }
};

namespace qlbm {

struct LatticeOps {
    cudaError_t (*step)(qlbm_ctx *h, bool odd);
    cudaError_t (*init_eq)(qlbm_ctx *h, const double *rho4, const double *u, const double *eps);
    cudaError_t (*get_state)(qlbm_ctx *h, double *out);
    cudaError_t (*set_state)(qlbm_ctx *h, const double *in);
    cudaError_t (*moments)(qlbm_ctx *h, double *rho4, double *u, double *eps);
    cudaError_t (*conserved_partial)(qlbm_ctx *h);
    // reverse mode (state buffers are natural-order copies with the layout of pop)
    cudaError_t (*adjoint)(qlbm_ctx *h, const void *state, const void *lam_in, void *lam_out);
    cudaError_t (*push)(qlbm_ctx *h, const void *src, void *dst);
    cudaError_t (*copy_natural)(qlbm_ctx *h, void *dst);
    cudaError_t (*lam_import)(qlbm_ctx *h, const double *in, void *lam);
    cudaError_t (*lam_export)(qlbm_ctx *h, const void *lam, double *out);
    cudaError_t (*init_adjoint)(qlbm_ctx *h, const double *lam, const double *rho4, const double *u,
                                const double *eps, double *grho4, double *gu, double *geps);
    // Fermi-Dirac parameter recovery (side output; FP64 step variant, NULL otherwise)
    cudaError_t (*fd_params)(qlbm_ctx *h, double *beta, double *mu_up, double *mu_dn, double *axis);
    cudaError_t (*step_fd)(qlbm_ctx *h, bool odd);
    cudaError_t (*fd_params_adjoint)(qlbm_ctx *h, const double *gbeta, const double *gmu_up,
                                     const double *gmu_dn, const double *gaxis, double *lam);
    cudaError_t (*init_fd)(qlbm_ctx *h, const double *beta, const double *mu_up, const double *mu_dn,
                           const double *axis, const double *u);
    // single-precision step that also writes the FD parameters (FP32 / FP16 storage; NULL otherwise)
    cudaError_t (*step_fdout)(qlbm_ctx *h, bool odd, float *beta, float *mu_up, float *mu_dn, float *axis);
    // negative-eigenvalue diagnostic of the equilibria of the current state (every precision)
    cudaError_t (*negative_eq)(qlbm_ctx *h, unsigned long long *count, unsigned *mask);
};

// Dispatch tables, one translation unit each (kernels_<lattice>_<codec>.cu).
const LatticeOps *ops_d2q9_fp64();
const LatticeOps *ops_d2q9_fp32();
const LatticeOps *ops_d2q9_fp16();
const LatticeOps *ops_d2q9_df64();
const LatticeOps *ops_d3q19_fp64();
const LatticeOps *ops_d3q19_fp32();
const LatticeOps *ops_d3q19_fp16();
const LatticeOps *ops_d3q19_df64();
const LatticeOps *ops_d2q9_fp64df();
const LatticeOps *ops_d3q19_fp64df();
// the double-float step on FP64 storage (kernels_<lattice>_fp64df.cu)
template <int D> cudaError_t step_f64df(qlbm_ctx *h, bool odd);

inline const LatticeOps *lattice_ops(int d, int prec)
{
    switch (prec) {
    case QLBM_FP64: return d == 2 ? ops_d2q9_fp64() : ops_d3q19_fp64();
    case QLBM_FP32: return d == 2 ? ops_d2q9_fp32() : ops_d3q19_fp32();
    case QLBM_FP16_DEV: return d == 2 ? ops_d2q9_fp16() : ops_d3q19_fp16();
    case QLBM_DF64: return d == 2 ? ops_d2q9_df64() : ops_d3q19_df64();
    case QLBM_FP64_DF: return d == 2 ? ops_d2q9_fp64df() : ops_d3q19_fp64df();
    default: return nullptr;
    }
}

cudaError_t launch_conserved_final(qlbm_ctx *h);

// Records the message returned by qlbm_last_error(NULL) for calls that have
// no handle; returns code.
int set_global_error(int code, const char *msg);

// Launch shape of the per-site kernels: one thread per site, blocks of up to
// kStepBlock consecutive x in one row.  Rows longer than 128 take the width
// among 128, 96 and 64 that leaves the fewest idle threads at the row's end
// (ties to the wider block): e.g. 96 for nx = 192, 64 for nx = 320.
inline int site_block_width(int nx)
{
    if (nx <= 128) return ((nx + 31) / 32) * 32;
    int best = 128, idle = (128 - nx % 128) % 128;
    for (int bx = 96; bx >= 64; bx -= 32) {
        const int id = (bx - nx % bx) % bx;
        if (id < idle) {
            best = bx;
            idle = id;
        }
    }
    return best;
}
inline dim3 site_block(const Grid &g) { return dim3(site_block_width(g.nx)); }
inline dim3 site_grid(const Grid &g, int bx)
{
    return dim3((unsigned)((int64_t)g.nxb * g.ny * g.nz));
}

// Rows per block of the row-pipelined step (k_step_aa_rows): rmax, or fewer
// where the grid would otherwise fall below four waves of resident blocks
// (the idle SMs of a short grid's last wave cost more than the pipelining
// gains).
inline int step_rows_per_block(const Grid &g, int rmax, int resident_per_sm, int sms)
{
    const int64_t blocks = (int64_t)g.nxb * g.ny * g.nz;
    const int64_t wave = (int64_t)resident_per_sm * (sms > 0 ? sms : 1);
    int64_t r = blocks / (4 * wave);
    if (r > rmax) r = rmax;
    return r < 1 ? 1 : (int)r;
}
inline dim3 row_group_grid(const Grid &g, int rpb)
{
    const int64_t rows = (int64_t)g.ny * g.nz;
    return dim3((unsigned)((int64_t)g.nxb * ((rows + rpb - 1) / rpb)));
}

}  // namespace qlbm
