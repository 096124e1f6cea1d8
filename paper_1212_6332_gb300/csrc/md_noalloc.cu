// Force evaluation for small systems that allocates no device memory.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// every device allocation through its own pool or memory cap, and
// latency-bound loops that must not enter the driver's allocator (which can
// synchronize the device and take unbounded time). md_forces_noalloc serves
// them: the caller passes positions and output buffers, and the only working
// memory is a fixed file-scope device array (g_noalloc_scratch) that every
// GPU loading this library holds until the process exits.
//
// The evaluation gives the forces and energies md_compute_forces gives (a
// density pass, F'(rho), a force pass) without cells or a neighbour list:
// positions are first wrapped into the box by the same rule (so unwrapped
// coordinates, any number of box lengths away, give the same result), then
// every thread loops over all atoms with the minimum-image convention,
// which is the right trade for the few thousand atoms this entry point is
// limited to.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "md.h"

namespace {

// Scratch (5 * MD_NOALLOC_MAX_ATOMS doubles, 640 KiB): F'(rho_i) at [0, n),
// E_i at [MAX, MAX + n), wrapped positions [n][3] at [2 MAX, 2 MAX + 3n).
constexpr int kScrE = MD_NOALLOC_MAX_ATOMS;
constexpr int kScrX = 2 * MD_NOALLOC_MAX_ATOMS;
__device__ __align__(256) double g_noalloc_scratch[5 * MD_NOALLOC_MAX_ATOMS];

constexpr int kNT = 128;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

struct PotS {
    int kind;
    double rc2, rs, rc, inv_w;
    double A2, xi2, p, p_r0, q2, q2_r0;  // RGL
    double eps, a, n, m, F_scale;        // SC
};

// x - L floor(x/L) with each operation rounded, folded into [0, L): the
// wrap md_compute_forces applies to its input positions.
__device__ __forceinline__ double na_wrap(double x, double L) {
    double k = floor(__ddiv_rn(x, L));
    double y = __dsub_rn(x, __dmul_rn(L, k));
    if (y < 0.0) y = __dadd_rn(y, L);
    if (y >= L) y = __dsub_rn(y, L);
    return y;
}

// minimum image of a separation of two wrapped coordinates (|d| < L)
__device__ __forceinline__ double mi(double d, double L) {
    double h = 0.5 * L;
    if (d > h) return d - L;
    if (d < -h) return d + L;
    return d;
}

// V, V', rho, rho' at r < rc (taper S = 1 - 10x^3 + 15x^4 - 6x^5)
__device__ __forceinline__ void pair_fn(const PotS& P, double r, double& V, double& dV, double& f, double& df) {
    double S = 1.0, dS = 0.0;
    if (r > P.rs) {
        double x = (r - P.rs) * P.inv_w;
        double x2 = x * x;
        S = 1.0 + x2 * x * (-10.0 + x * (15.0 - 6.0 * x));
        dS = x2 * (-30.0 + x * (60.0 - 30.0 * x)) * P.inv_w;
    }
    if (P.kind == MD_POT_RGL) {
        double e1 = P.A2 * exp(P.p - P.p_r0 * r);
        double e2 = P.xi2 * exp(P.q2 - P.q2_r0 * r);
        V = e1 * S;
        dV = e1 * (dS - P.p_r0 * S);
        f = e2 * S;
        df = e2 * (dS - P.q2_r0 * S);
    } else {
        double an = P.eps * pow(P.a / r, P.n), am = pow(P.a / r, P.m);
        V = an * S;
        dV = an * (dS - P.n / r * S);
        f = am * S;
        df = am * (dS - P.m / r * S);
    }
}

__global__ void __launch_bounds__(kNT) k_na_wrap(int n, const double* __restrict__ x_in, double Lx, double Ly,
                                                 double Lz, double* __restrict__ scratch) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double* x = scratch + kScrX;
    x[3 * i] = na_wrap(x_in[3 * i], Lx);
    x[3 * i + 1] = na_wrap(x_in[3 * i + 1], Ly);
    x[3 * i + 2] = na_wrap(x_in[3 * i + 2], Lz);
}

__global__ void __launch_bounds__(kNT) k_na_density(int n, double Lx, double Ly, double Lz, PotS P,
                                                    double* __restrict__ scratch) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* x = scratch + kScrX;
    double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    double rho = 0.0, ep = 0.0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = mi(x[3 * j] - xi, Lx), dy = mi(x[3 * j + 1] - yi, Ly), dz = mi(x[3 * j + 2] - zi, Lz);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.rc2) continue;
        double V, dV, f, df;
        pair_fn(P, sqrt(r2), V, dV, f, df);
        rho += f;
        ep += V;
    }
    double F = 0.0, Fp = 0.0;
    if (rho > 0.0) {
        double s = sqrt(rho);
        F = -P.F_scale * s;
        Fp = -0.5 * P.F_scale / s;
    }
    scratch[i] = Fp;
    scratch[kScrE + i] = F + 0.5 * ep;
}

__global__ void __launch_bounds__(kNT) k_na_force(int n, double Lx, double Ly, double Lz, PotS P,
                                                  const double* __restrict__ scratch, double* __restrict__ f_out,
                                                  double* __restrict__ e_atom) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* x = scratch + kScrX;
    double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    double Fpi = scratch[i];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        double dx = mi(x[3 * j] - xi, Lx), dy = mi(x[3 * j + 1] - yi, Ly), dz = mi(x[3 * j + 2] - zi, Lz);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= P.rc2) continue;
        double r = sqrt(r2);
        double V, dV, f, df;
        pair_fn(P, r, V, dV, f, df);
        double s = (dV + (Fpi + scratch[j]) * df) / r;
        fx += s * dx;
        fy += s * dy;
        fz += s * dz;
    }
    f_out[3 * i] = fx;
    f_out[3 * i + 1] = fy;
    f_out[3 * i + 2] = fz;
    if (e_atom) e_atom[i] = scratch[kScrE + i];
}

// One block sums E_i in a fixed order (deterministic).
__global__ void __launch_bounds__(1024) k_na_total(int n, const double* __restrict__ scratch, double* e_total) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) s += scratch[kScrE + i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 32; ++k) t += sh[k];
        *e_total = t;
    }
}

// Device memory of device `dev` (the current one), or managed memory.
bool dev_ptr(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" {

int md_forces_noalloc(const md_potential* pot, const double* box, int64_t n_atoms, const double* x, double* f,
                      double* e_atom, double* e_total, md_stream stream) {
    if (!pot || !box) return MD_ERR_ARG;  // potential or box is NULL
    if (n_atoms < 0) return MD_ERR_ARG;  // n_atoms must be >= 0
    if (n_atoms > MD_NOALLOC_MAX_ATOMS) return MD_ERR_ARG;  // beyond the fixed scratch
    if (pot->kind != MD_POT_RGL && pot->kind != MD_POT_SC)
        return MD_ERR_UNSUPPORTED;  // md_forces_noalloc supports the RGL and Sutton-Chen potentials
    for (int k = 0; k < 5; ++k)
        if (!std::isfinite(pot->p[k])) return MD_ERR_ARG;  // non-finite potential parameter
    if (!(pot->r_cut > 0.0) || !std::isfinite(pot->r_cut) || !std::isfinite(pot->r_taper))
        return MD_ERR_ARG;  // r_cut must be positive and finite
    if (pot->kind == MD_POT_RGL && !(pot->p[4] > 0.0)) return MD_ERR_ARG;  // RGL r0 must be positive
    if (pot->kind == MD_POT_SC && !(pot->p[2] > 0.0)) return MD_ERR_ARG;  // Sutton-Chen a must be positive
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0.0) || !std::isfinite(box[a]) || !(pot->r_cut < 0.5 * box[a]))
            return MD_ERR_ARG;  // box lengths must exceed twice r_cut (minimum image)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return MD_ERR_CUDA;  // cudaGetDevice failed
    }
    // x and f may be NULL only when there are no atoms; every pointer given
    // must be device (or managed) memory of the current device
    if (n_atoms > 0 && (!x || !f)) return MD_ERR_ARG;  // x and f are required
    if ((x && !dev_ptr(x, dev)) || (f && !dev_ptr(f, dev)) || (e_atom && !dev_ptr(e_atom, dev)) ||
        (e_total && !dev_ptr(e_total, dev)))
        return MD_ERR_ARG;  // x, f, e_atom, e_total must be memory of the current device
    cudaStream_t s = (cudaStream_t)stream;
    if (n_atoms == 0) {
        // no atoms: E_T = 0 (a memset enqueued on the stream, no allocation)
        if (e_total && cudaMemsetAsync(e_total, 0, sizeof(double), s) != cudaSuccess) {
            cudaGetLastError();
            return MD_ERR_CUDA;  // the memset could not be enqueued
        }
        return MD_OK;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            // once per device, with that device current: the host-side name of
            // the array is not a device address, so ask the runtime for it
            cudaError_t ce = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_noalloc_scratch);
            if (ce != cudaSuccess) {
                g_scratch_ptr[dev] = nullptr;
                return MD_ERR_CUDA;  // the runtime could not resolve the array
            }
        }
        scratch = g_scratch_ptr[dev];
    }

    PotS P{};
    P.kind = pot->kind;
    P.rc = pot->r_cut;
    P.rc2 = pot->r_cut * pot->r_cut;
    if (pot->r_taper < pot->r_cut) {
        P.rs = pot->r_taper;
        P.inv_w = 1.0 / (pot->r_cut - pot->r_taper);
    } else {
        P.rs = pot->r_cut;
        P.inv_w = 0.0;
    }
    P.F_scale = 1.0;
    if (pot->kind == MD_POT_RGL) {
        P.A2 = 2.0 * pot->p[0];
        P.xi2 = pot->p[1] * pot->p[1];
        P.p = pot->p[2];
        P.p_r0 = pot->p[2] / pot->p[4];
        P.q2 = 2.0 * pot->p[3];
        P.q2_r0 = 2.0 * pot->p[3] / pot->p[4];
    } else {
        P.eps = pot->p[0];
        P.a = pot->p[2];
        P.n = pot->p[3];
        P.m = pot->p[4];
        P.F_scale = pot->p[1] * pot->p[0];
    }
    int n = (int)n_atoms;
    int nb = (n + kNT - 1) / kNT;
    k_na_wrap<<<nb, kNT, 0, s>>>(n, x, box[0], box[1], box[2], scratch);
    k_na_density<<<nb, kNT, 0, s>>>(n, box[0], box[1], box[2], P, scratch);
    k_na_force<<<nb, kNT, 0, s>>>(n, box[0], box[1], box[2], P, scratch, f, e_atom);
    if (e_total) k_na_total<<<1, 1024, 0, s>>>(n, scratch, e_total);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return MD_ERR_CUDA;  // a launch failed
    return MD_OK;
}

}  // extern "C"
