// Differentiable OBC generalized-Born energy of a batch of configurations:
// cph_gb_energy (forward) and cph_gb_energy_backward (adjoint with respect to
// positions, charges and intrinsic radii).  The model is the one the paper
// names for its implicit-solvent runs (OBC "igb=2", Implicit Solvent
// Calculations section); E_GB = -1/2 k tau sum_i sum_j q_i q_j / f_ij over all
// pairs including i = j (f_ii = R_i), tau = 1/eps_in - 1/eps_out.
//
// Layout: replica r, atom a -> index r*n + a; x is [n_rep][n][3] float.
// One CTA of kTile threads owns one (replica, i-tile); every ordered pair is
// evaluated by the owner of i (no atomics except the per-replica energy sum).
//
// Gradient with respect to rho_i (rt = rho - offset, s = screen * rt enter
// every descreening integral H(r, rt_i, s_j) of psi_i = rt_i/2 sum_j H):
//   dE/drho_i = dE/dR_i R_i^2 (1/rt_i^2 - tanh(theta_i)/rho_i^2)     [R_i, psi fixed]
//             + g_i psi_i / rt_i                                    [psi_i = rt_i I_i]
//             + c_i sum_j dH(r_ij; rt_i, s_j)/drt                   [own integrals]
//             + screen_i sum_j c_j dH(r_ij; rt_j, s_i)/ds           [partners' integrals]
// with g_i = dE/dR_i dR_i/dpsi_i and c_i = g_i rt_i / 2.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/cphremd.h"
#include "cph_device.cuh"

namespace cph {
namespace grad {

constexpr int kT = 128;
constexpr float kFar = 1.0e4f;

struct GView {
    int n_rep, n, ntile;
    const float *x, *q, *rho, *screen;
    double tau, sqrt_k, alpha, beta, gamma, offset;
    // workspace, per replica-atom
    double *psi, *R, *dRdpsi, *dEdR, *c, *dxd, *dqa;
    long long* eacc; // [n_rep]
    double* E;
    const double* dE;
    float *dx, *dq, *drho;
};

// workspace layout (bytes, each region 256-aligned)
inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

inline size_t ws_bytes(long long n_rep, long long n) {
    const size_t na = (size_t)(n_rep * n);
    return 6 * align256(na * sizeof(double)) + align256(3 * na * sizeof(double)) +
           align256((size_t)n_rep * sizeof(long long));
}

inline void ws_carve(GView& g, void* base) {
    char* p = (char*)base;
    const size_t na = (size_t)g.n_rep * g.n;
    double** d1[] = {&g.psi, &g.R, &g.dRdpsi, &g.dEdR, &g.c, &g.dqa};
    for (double** d : d1) {
        *d = (double*)p;
        p += align256(na * sizeof(double));
    }
    g.dxd = (double*)p;
    p += align256(3 * na * sizeof(double));
    g.eacc = (long long*)p;
}

struct alignas(16) F4 {
    float x, y, z, w;
};

__global__ void __launch_bounds__(kT) k_born(GView g) {
    __shared__ F4 sj[kT];
    const int rep = blockIdx.x / g.ntile, i0 = (blockIdx.x % g.ntile) * kT;
    const int tid = threadIdx.x, i = i0 + tid, n = g.n;
    const bool vi = i < n;
    const float* X = g.x + (size_t)rep * n * 3;
    const float* RH = g.rho + (size_t)rep * n;
    if (i0 == 0 && tid == 0) g.eacc[rep] = 0;
    const float cx = X[3 * i0], cy = X[3 * i0 + 1], cz = X[3 * i0 + 2];
    float xi = -kFar, yi = -kFar, zi = -kFar, rti = 1.f;
    if (vi) {
        xi = X[3 * i] - cx;
        yi = X[3 * i + 1] - cy;
        zi = X[3 * i + 2] - cz;
        rti = RH[i] - (float)g.offset;
    }
    const float irti = 1.f / rti;
    long long acc = 0;
    const int tself = i0 / kT;
    for (int j0 = 0, jt = 0; j0 < n; j0 += kT, ++jt) {
        __syncthreads();
        const int j = j0 + tid;
        F4 v;
        if (j < n) {
            v.x = X[3 * j] - cx;
            v.y = X[3 * j + 1] - cy;
            v.z = X[3 * j + 2] - cz;
            v.w = g.screen[j] * (RH[j] - (float)g.offset);
        } else {
            v.x = v.y = v.z = kFar;
            v.w = 0.f;
        }
        sj[tid] = v;
        __syncthreads();
        float part = 0.f;
        if (jt != tself) {
#pragma unroll 4
            for (int k = 0; k < kT; ++k) {
                const F4 b = sj[k];
                const float dx = xi - b.x, dy = yi - b.y, dz = zi - b.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float rinv = rsqrt_ftz(r2);
                part += hct(r2 * rinv, rinv, rti, irti, b.w);
            }
        } else {
            for (int k = 0; k < kT; ++k) {
                const F4 b = sj[k];
                const bool self = (k == tid);
                const float dx = xi - b.x, dy = yi - b.y, dz = zi - b.z;
                float r2 = dx * dx + dy * dy + dz * dz;
                r2 = self ? 1.f : r2;
                const float rinv = rsqrt_ftz(r2);
                const float h = hct(r2 * rinv, rinv, rti, irti, b.w);
                part += self ? 0.f : h;
            }
        }
        acc += to_fixed(part, (float)kScaleH);
    }
    if (vi) {
        const size_t a = (size_t)rep * n + i;
        const double rt = (double)RH[i] - g.offset, rho = RH[i];
        const double psi = 0.5 * rt * ((double)acc / kScaleH);
        const double th = tanh(psi * (g.alpha + psi * (-g.beta + psi * g.gamma)));
        const double R = 1.0 / (1.0 / rt - th / rho);
        g.psi[a] = psi;
        g.R[a] = R;
        g.dRdpsi[a] = R * R * (1.0 - th * th) * (g.alpha + psi * (-2.0 * g.beta + 3.0 * g.gamma * psi)) / rho;
    }
}

template <bool BACKWARD>
__global__ void __launch_bounds__(kT) k_pair(GView g) {
    __shared__ F4 sa[kT];
    __shared__ F4 sb[kT];
    __shared__ long long red[4];
    const int rep = blockIdx.x / g.ntile, i0 = (blockIdx.x % g.ntile) * kT;
    const int tid = threadIdx.x, i = i0 + tid, n = g.n;
    const bool vi = i < n;
    const float* X = g.x + (size_t)rep * n * 3;
    const float* Q = g.q + (size_t)rep * n;
    const size_t base = (size_t)rep * n;
    const float sqk = (float)g.sqrt_k, tau = (float)g.tau;
    const float cx = X[3 * i0], cy = X[3 * i0 + 1], cz = X[3 * i0 + 2];
    float xi = -kFar, yi = -kFar, zi = -kFar, qi = 0.f, Ri = 1.f, iRi = 1.f;
    if (vi) {
        xi = X[3 * i] - cx;
        yi = X[3 * i + 1] - cy;
        zi = X[3 * i + 2] - cz;
        qi = Q[i] * sqk;
        Ri = (float)g.R[base + i];
        iRi = (float)(1.0 / g.R[base + i]);
    }
    long long egb = 0, adr = 0, aq = 0, gx = 0, gy = 0, gz = 0;
    const int tself = i0 / kT;
    for (int j0 = 0, jt = 0; j0 < n; j0 += kT, ++jt) {
        __syncthreads();
        const int j = j0 + tid;
        F4 a, b;
        if (j < n) {
            a.x = X[3 * j] - cx;
            a.y = X[3 * j + 1] - cy;
            a.z = X[3 * j + 2] - cz;
            a.w = Q[j] * sqk;
            b.x = (float)g.R[base + j];
            b.y = (float)(1.0 / g.R[base + j]);
        } else {
            a.x = a.y = a.z = kFar;
            a.w = 0.f;
            b.x = b.y = 1.f;
        }
        b.z = b.w = 0.f;
        sa[tid] = a;
        sb[tid] = b;
        __syncthreads();
        KSum<float> pe;
        float pdr = 0.f, pq = 0.f, px = 0.f, py = 0.f, pz = 0.f;
        const bool diag = (jt == tself);
#pragma unroll 2
        for (int k = 0; k < kT; ++k) {
            const F4 A = sa[k];
            const F4 B = sb[k];
            const bool self = diag && (k == tid);
            const float dx = xi - A.x, dy = yi - A.y, dz = zi - A.z;
            float r2 = dx * dx + dy * dy + dz * dz;
            r2 = self ? 1.f : r2;
            const float m = self ? 0.f : 1.f;
            const float D = 0.25f * r2 * (iRi * B.y);
            const float e = exp2_ftz(-D * kLog2e);
            const float fi = m * rsqrt_ftz(r2 + (Ri * B.x) * e);
            pe.add(qi * A.w * fi);
            if (BACKWARD) {
                const float qf3 = qi * A.w * fi * fi * fi;
                pdr += qf3 * B.x * e * (1.f + D);
                pq += A.w * fi;
                const float t = tau * qf3 * (1.f - 0.25f * e);
                px += t * dx;
                py += t * dy;
                pz += t * dz;
            }
        }
        egb += to_fixed(pe.value(), (float)kScaleE);
        if (BACKWARD) {
            adr += to_fixed(pdr, (float)kScaleE);
            aq += to_fixed(pq, (float)kScaleE);
            gx += to_fixed(px, (float)kScaleE);
            gy += to_fixed(py, (float)kScaleE);
            gz += to_fixed(pz, (float)kScaleE);
        }
    }
    long long ei = 0;
    if (vi) {
        const double q = (double)Q[i] * g.sqrt_k, R = g.R[base + i];
        ei = __double2ll_rn(-0.5 * g.tau * ((double)egb / kScaleE + q * q / R) * kScaleE);
        if (BACKWARD) {
            const size_t a = base + i;
            const double dEdR = 0.5 * g.tau * ((double)adr / kScaleE + q * q / (R * R));
            const double rt = (double)g.rho[a] - g.offset;
            g.dEdR[a] = dEdR;
            g.c[a] = dEdR * g.dRdpsi[a] * 0.5 * rt;
            g.dqa[a] = -g.tau * g.sqrt_k * ((double)aq / kScaleE + q / R);
            g.dxd[3 * a] = (double)gx / kScaleE;
            g.dxd[3 * a + 1] = (double)gy / kScaleE;
            g.dxd[3 * a + 2] = (double)gz / kScaleE;
        }
    }
    // per-replica energy (fixed-order block sum, then one int64 atomic)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ei += __shfl_down_sync(0xffffffffu, ei, o);
    if ((tid & 31) == 0) red[tid >> 5] = ei;
    __syncthreads();
    if (tid == 0) atomicAdd((unsigned long long*)&g.eacc[rep], (unsigned long long)(red[0] + red[1] + red[2] + red[3]));
}

__global__ void __launch_bounds__(kT) k_chain(GView g) {
    __shared__ F4 sa[kT];
    __shared__ F4 sb[kT];
    const int rep = blockIdx.x / g.ntile, i0 = (blockIdx.x % g.ntile) * kT;
    const int tid = threadIdx.x, i = i0 + tid, n = g.n;
    const bool vi = i < n;
    const float* X = g.x + (size_t)rep * n * 3;
    const float* RH = g.rho + (size_t)rep * n;
    const size_t base = (size_t)rep * n;
    const float cx = X[3 * i0], cy = X[3 * i0 + 1], cz = X[3 * i0 + 2];
    float xi = -kFar, yi = -kFar, zi = -kFar, ci = 0.f, si = 0.f, rti = 1.f;
    if (vi) {
        xi = X[3 * i] - cx;
        yi = X[3 * i + 1] - cy;
        zi = X[3 * i + 2] - cz;
        ci = (float)g.c[base + i];
        rti = RH[i] - (float)g.offset;
        si = g.screen[i] * rti;
    }
    const float irti = 1.f / rti;
    long long gx = 0, gy = 0, gz = 0, art = 0, as = 0;
    const int tself = i0 / kT;
    for (int j0 = 0, jt = 0; j0 < n; j0 += kT, ++jt) {
        __syncthreads();
        const int j = j0 + tid;
        F4 a, b;
        if (j < n) {
            a.x = X[3 * j] - cx;
            a.y = X[3 * j + 1] - cy;
            a.z = X[3 * j + 2] - cz;
            a.w = (float)g.c[base + j];
            b.y = RH[j] - (float)g.offset;
            b.x = g.screen[j] * b.y;
        } else {
            a.x = a.y = a.z = kFar;
            a.w = 0.f;
            b.x = 0.f;
            b.y = 1.f;
        }
        b.z = b.w = 0.f;
        sa[tid] = a;
        sb[tid] = b;
        __syncthreads();
        float px = 0.f, py = 0.f, pz = 0.f, prt = 0.f, ps = 0.f;
        const bool diag = (jt == tself);
#pragma unroll 2
        for (int k = 0; k < kT; ++k) {
            const F4 A = sa[k];
            const F4 B = sb[k];
            const bool self = diag && (k == tid);
            const float dx = xi - A.x, dy = yi - A.y, dz = zi - A.z;
            float r2 = dx * dx + dy * dy + dz * dz;
            r2 = self ? 1.f : r2;
            const float m = self ? 0.f : 1.f;
            const float rinv = rsqrt_ftz(r2);
            const float r = r2 * rinv;
            const float gr = ci * hct_dr(r, rinv, rti, B.x) + A.w * hct_dr(r, rinv, B.y, si);
            const float t = m * gr * rinv;
            px += t * dx;
            py += t * dy;
            pz += t * dz;
            prt += m * hct_drt(r, rti, irti, B.x);
            ps += m * A.w * hct_ds(r, rinv, B.y, si);
        }
        gx += to_fixed(px, (float)kScaleE);
        gy += to_fixed(py, (float)kScaleE);
        gz += to_fixed(pz, (float)kScaleE);
        art += to_fixed(prt, (float)kScaleE);
        as += to_fixed(ps, (float)kScaleE);
    }
    if (vi) {
        const size_t a = base + i;
        const double up = g.dE[rep];
        const double rho = RH[i], rt = rho - g.offset, R = g.R[a], psi = g.psi[a];
        const double th = tanh(psi * (g.alpha + psi * (-g.beta + psi * g.gamma)));
        const double dEdR = g.dEdR[a];
        const double gpsi = dEdR * g.dRdpsi[a];
        const double c = g.c[a];
        double dr = dEdR * R * R * (1.0 / (rt * rt) - th / (rho * rho)) + gpsi * psi / rt +
                    c * ((double)art / kScaleE) + (double)g.screen[i] * ((double)as / kScaleE);
        g.dx[3 * a] = (float)(up * (g.dxd[3 * a] + (double)gx / kScaleE));
        g.dx[3 * a + 1] = (float)(up * (g.dxd[3 * a + 1] + (double)gy / kScaleE));
        g.dx[3 * a + 2] = (float)(up * (g.dxd[3 * a + 2] + (double)gz / kScaleE));
        g.dq[a] = (float)(up * g.dqa[a]);
        g.drho[a] = (float)(up * dr);
    }
}

__global__ void k_energy_out(GView g) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < g.n_rep) g.E[r] = (double)g.eacc[r] / kScaleE;
}

} // namespace grad
} // namespace cph

using namespace cph;
using namespace cph::grad;

void cph_internal_set_error(const std::string& m);

namespace {
int gfail(int code, const std::string& m) {
    cph_internal_set_error(m);
    return code;
}

int setup(GView& g, int n_rep, int n, const float* x, const float* q, const float* rho,
          const float* screen, const cph_gb_params* gb, void* ws, size_t wsb) {
    if (n_rep < 1 || n < 1 || !x || !q || !rho || !screen || !gb || !ws)
        return gfail(CPH_E_INVALID, "cph_gb_energy: bad arguments");
    if ((size_t)n_rep * (size_t)n > (size_t)1 << 31) return gfail(CPH_E_INVALID, "cph_gb_energy: too many atoms");
    if (((uintptr_t)ws & 255u) != 0) return gfail(CPH_E_INVALID, "cph_gb_energy: workspace must be 256-byte aligned");
    if (wsb < ws_bytes(n_rep, n)) return gfail(CPH_E_INVALID, "cph_gb_energy: workspace too small");
    if (!(gb->eps_in > 0) || !(gb->eps_out > 0)) return gfail(CPH_E_INVALID, "cph_gb_energy: bad dielectric");
    g = GView{};
    g.n_rep = n_rep;
    g.n = n;
    g.ntile = (n + kT - 1) / kT;
    g.x = x;
    g.q = q;
    g.rho = rho;
    g.screen = screen;
    g.tau = 1.0 / gb->eps_in - 1.0 / gb->eps_out;
    g.sqrt_k = std::sqrt(kCoulomb);
    g.alpha = gb->alpha;
    g.beta = gb->beta;
    g.gamma = gb->gamma;
    g.offset = gb->offset;
    ws_carve(g, ws);
    return CPH_OK;
}
} // namespace

extern "C" size_t cph_gb_workspace_bytes(int n_rep, int n) {
    if (n_rep < 1 || n < 1) return 0;
    return ws_bytes(n_rep, n);
}

extern "C" int cph_gb_energy(int n_rep, int n, const float* x, const float* q, const float* rho,
                             const float* screen, const cph_gb_params* gb, double* E, void* ws,
                             size_t wsb, void* stream) {
    GView g;
    int rc = setup(g, n_rep, n, x, q, rho, screen, gb, ws, wsb);
    if (rc != CPH_OK) return rc;
    if (!E) return gfail(CPH_E_INVALID, "cph_gb_energy: E is NULL");
    g.E = E;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = n_rep * g.ntile;
    k_born<<<grid, kT, 0, st>>>(g);
    k_pair<false><<<grid, kT, 0, st>>>(g);
    k_energy_out<<<(n_rep + 127) / 128, 128, 0, st>>>(g);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return gfail(CPH_E_CUDA, std::string("cph_gb_energy: ") + cudaGetErrorString(ce));
    return CPH_OK;
}

extern "C" int cph_gb_energy_backward(int n_rep, int n, const float* x, const float* q,
                                      const float* rho, const float* screen,
                                      const cph_gb_params* gb, const double* dE, float* dx,
                                      float* dq, float* drho, void* ws, size_t wsb, void* stream) {
    GView g;
    int rc = setup(g, n_rep, n, x, q, rho, screen, gb, ws, wsb);
    if (rc != CPH_OK) return rc;
    if (!dE || !dx || !dq || !drho) return gfail(CPH_E_INVALID, "cph_gb_energy_backward: NULL output");
    g.dE = dE;
    g.dx = dx;
    g.dq = dq;
    g.drho = drho;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = n_rep * g.ntile;
    k_born<<<grid, kT, 0, st>>>(g);
    k_pair<true><<<grid, kT, 0, st>>>(g);
    k_chain<<<grid, kT, 0, st>>>(g);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return gfail(CPH_E_CUDA, std::string("cph_gb_energy_backward: ") + cudaGetErrorString(ce));
    return CPH_OK;
}

// ---------------------------------------------------------------------------
// cph_gb_energy_noalloc: the forward GB energy with its scratch in a fixed
// file-scope device array instead of a caller workspace.  Host code only sees
// a host-side stand-in for g_gb_noalloc_scratch: its device address is looked
// up per device with cudaGetSymbolAddress (with that device current) and
// cached; the kernels receive that address.
namespace {
static __device__ __align__(256) unsigned char g_gb_noalloc_scratch[CPH_GB_NOALLOC_SCRATCH_BYTES];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

int noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return gfail(CPH_E_CUDA, std::string("cph_gb_energy_noalloc: cudaGetDevice: ") + cudaGetErrorString(ce));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return gfail(CPH_E_INVALID, "cph_gb_energy_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        ce = cudaGetSymbolAddress(&p, g_gb_noalloc_scratch);
        if (ce != cudaSuccess || !p)
            return gfail(CPH_E_CUDA, std::string("cph_gb_energy_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return CPH_OK;
}
} // namespace

extern "C" int cph_gb_energy_noalloc(int n_rep, int n, const float* x, const float* q, const float* rho,
                                     const float* screen, const cph_gb_params* gb, double* E, void* stream) {
    if (n_rep < 1 || n < 1) return gfail(CPH_E_INVALID, "cph_gb_energy_noalloc: bad sizes");
    const size_t need = ws_bytes(n_rep, n);
    if (need > CPH_GB_NOALLOC_SCRATCH_BYTES)
        return gfail(CPH_E_INVALID, "cph_gb_energy_noalloc: n_rep * n too large: needs " + std::to_string(need) +
                                        " bytes of scratch, the fixed array holds " +
                                        std::to_string((size_t)CPH_GB_NOALLOC_SCRATCH_BYTES));
    void* ws = nullptr;
    int rc = noalloc_scratch(&ws);
    if (rc != CPH_OK) return rc;
    return cph_gb_energy(n_rep, n, x, q, rho, screen, gb, E, ws, CPH_GB_NOALLOC_SCRATCH_BYTES, stream);
}
