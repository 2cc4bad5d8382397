// Differentiable OBC generalized-Born energy of a batch of configurations:
// cph_gb_energy (forward) and cph_gb_energy_backward (adjoint with respect to
// positions, charges and intrinsic radii).  The model is the one the paper
// names for its implicit-solvent runs (OBC "igb=2", Implicit Solvent
// Calculations section); E_GB = -1/2 k tau sum_i sum_j q_i q_j / f_ij over all
// pairs including i = j (f_ii = R_i), tau = 1/eps_in - 1/eps_out.
//
// Layout: replica r, atom a -> index r*n + a; x is [n_rep][n][3] float.
// Kernels: cph_grad_sym.cuh (each unordered pair evaluated once, int64
// fixed-point accumulation in the caller's workspace).
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
#include "cph_grad_sym.cuh"

namespace cph {
namespace grad {

// Workspace: eleven 8-byte slots per replica-atom, the per-replica energy sums
// and the two-word far-pair bound, each region 256-byte aligned.  Slots that
// are never live together share memory:
//   0 psi | 1 R | 2 Hfix -> dRfix -> dE/dR | 3 dR/dpsi -> dE/dpsi | 4 c
//   5 dqfix -> dE/dq | 6-8 gradient (fixed point) | 9 art | 10 as
constexpr int kSlots = 11;

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

inline size_t ws_bytes(long long n_rep, long long n) {
    const size_t na = (size_t)(n_rep * n);
    return 8 * align256(na * sizeof(double)) + align256(3 * na * sizeof(double)) +
           align256((size_t)n_rep * sizeof(long long)) + 256;
}

inline void ws_carve_sym(SView& g, void* base) {
    char* p = (char*)base;
    const size_t na = (size_t)g.n_rep * g.n;
    const size_t sl = align256(na * sizeof(double));
    g.psi = (double*)p;
    g.R = (double*)(p + sl);
    g.Hfix = g.dRfix = (long long*)(p + 2 * sl);
    g.dEdR = (double*)(p + 2 * sl);
    g.gpsi = (double*)(p + 3 * sl);
    g.c = (double*)(p + 4 * sl);
    g.dqfix = (long long*)(p + 5 * sl);
    g.dq = (double*)(p + 5 * sl);
    g.gfix = (long long*)(p + 6 * sl);
    const size_t s3 = align256(3 * na * sizeof(double));
    g.artfix = (long long*)(p + 6 * sl + s3);
    g.asfix = (long long*)(p + 7 * sl + s3);
    g.eacc = (long long*)(p + 8 * sl + s3);
    g.bound = (unsigned int*)(p + 8 * sl + s3 + align256((size_t)g.n_rep * sizeof(long long)));
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

int setup(SView& g, int n_rep, int n, const float* x, const float* q, const float* rho,
          const float* screen, const cph_gb_params* gb, void* ws, size_t wsb) {
    if (n_rep < 1 || n < 1 || !x || !q || !rho || !screen || !gb || !ws)
        return gfail(CPH_E_INVALID, "cph_gb_energy: bad arguments");
    if ((size_t)n_rep * (size_t)n > (size_t)1 << 31) return gfail(CPH_E_INVALID, "cph_gb_energy: too many atoms");
    if (((uintptr_t)ws & 255u) != 0) return gfail(CPH_E_INVALID, "cph_gb_energy: workspace must be 256-byte aligned");
    if (wsb < ws_bytes(n_rep, n)) return gfail(CPH_E_INVALID, "cph_gb_energy: workspace too small");
    if (!(gb->eps_in > 0) || !(gb->eps_out > 0)) return gfail(CPH_E_INVALID, "cph_gb_energy: bad dielectric");
    if (!std::isfinite(gb->sa_gamma) || !(gb->sa_probe >= 0))
        return gfail(CPH_E_INVALID, "cph_gb_energy: bad surface-term parameters");
    if (!(gb->kappa >= 0) || !std::isfinite(gb->kappa))
        return gfail(CPH_E_INVALID, "cph_gb_energy: salt screening kappa must be finite and >= 0");
    if (!(gb->rgbmax >= 0) || !std::isfinite(gb->rgbmax))
        return gfail(CPH_E_INVALID, "cph_gb_energy: rgbmax must be finite and >= 0 (0 = no cutoff)");
    g = SView{};
    g.n_rep = n_rep;
    g.n = n;
    g.n_itile = (n + kGI - 1) / kGI;
    g.n_jtile = (n + kGJ - 1) / kGJ;
    g.n_chunk = (g.n_jtile + kGChunk - 1) / kGChunk;
    g.x = x;
    g.q = q;
    g.rho = rho;
    g.screen = screen;
    g.tau = 1.0 / gb->eps_in - 1.0 / gb->eps_out;
    g.kappa = gb->kappa;
    g.inv_eps_in = 1.0 / gb->eps_in;
    g.inv_eps_out = 1.0 / gb->eps_out;
    g.tau_pair = gb->kappa > 0 ? 1.0 : g.tau;
    g.sqrt_k = std::sqrt(kCoulomb);
    g.alpha = gb->alpha;
    g.beta = gb->beta;
    g.gamma = gb->gamma;
    g.offset = gb->offset;
    g.sa_gamma = gb->sa_gamma;
    g.sa_probe = gb->sa_probe;
    g.rgbmax = gb->rgbmax > 0 ? gb->rgbmax : INFINITY;
    g.tau32 = (float)g.tau;
    g.sqk32 = (float)g.sqrt_k;
    g.iei32 = (float)g.inv_eps_in;
    g.ieo32 = (float)g.inv_eps_out;
    g.kap32 = (float)g.kappa;
    g.off32 = (float)g.offset;
    g.rgbmax32 = (float)g.rgbmax;
    ws_carve_sym(g, ws);
    return CPH_OK;
}

// bound and Born radii, shared by both directions
int launch_radii(SView& g, cudaStream_t st) {
    const size_t na = (size_t)g.n_rep * g.n;
    cudaError_t ce = cudaMemsetAsync(g.bound, 0, 2 * sizeof(unsigned int), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g.Hfix, 0, na * sizeof(long long), st);
    if (ce != cudaSuccess) return gfail(CPH_E_CUDA, std::string("cph_gb_energy: memset: ") + cudaGetErrorString(ce));
    const int ba = (int)((na + 255) / 256);
    const int grid = g.n_rep * g.n_itile * g.n_chunk;
    k_gbound<<<ba, 256, 0, st>>>(g);
    if (g.rgbmax < INFINITY) k_gborn_sym<true><<<grid, kGT, 0, st>>>(g);
    else k_gborn_sym<false><<<grid, kGT, 0, st>>>(g);
    k_gfin_born<<<ba, 256, 0, st>>>(g);
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
    SView g;
    int rc = setup(g, n_rep, n, x, q, rho, screen, gb, ws, wsb);
    if (rc != CPH_OK) return rc;
    if (!E) return gfail(CPH_E_INVALID, "cph_gb_energy: E is NULL");
    g.E = E;
    cudaStream_t st = (cudaStream_t)stream;
    rc = launch_radii(g, st);
    if (rc != CPH_OK) return rc;
    const size_t na = (size_t)n_rep * n;
    const int ba = (int)((na + 255) / 256);
    if (g.kappa > 0) k_gpair_sym<false, true><<<n_rep * g.n_itile * g.n_chunk, kGT, 0, st>>>(g);
    else k_gpair_sym<false, false><<<n_rep * g.n_itile * g.n_chunk, kGT, 0, st>>>(g);
    k_gfin_c<false><<<ba, 256, 0, st>>>(g);
    k_genergy_out<<<(n_rep + 127) / 128, 128, 0, st>>>(g);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return gfail(CPH_E_CUDA, std::string("cph_gb_energy: ") + cudaGetErrorString(ce));
    return CPH_OK;
}

extern "C" int cph_gb_energy_backward(int n_rep, int n, const float* x, const float* q,
                                      const float* rho, const float* screen,
                                      const cph_gb_params* gb, const double* dE, float* dx,
                                      float* dq, float* drho, void* ws, size_t wsb, void* stream) {
    SView g;
    int rc = setup(g, n_rep, n, x, q, rho, screen, gb, ws, wsb);
    if (rc != CPH_OK) return rc;
    if (!dE || !dx || !dq || !drho) return gfail(CPH_E_INVALID, "cph_gb_energy_backward: NULL output");
    g.dE = dE;
    g.dx = dx;
    g.dqo = dq;
    g.drho = drho;
    cudaStream_t st = (cudaStream_t)stream;
    rc = launch_radii(g, st);
    if (rc != CPH_OK) return rc;
    const size_t na = (size_t)n_rep * n;
    const int ba = (int)((na + 255) / 256);
    const int grid = n_rep * g.n_itile * g.n_chunk;
    if (g.kappa > 0) k_gpair_sym<true, true><<<grid, kGT, 0, st>>>(g);
    else k_gpair_sym<true, false><<<grid, kGT, 0, st>>>(g);
    k_gfin_c<true><<<ba, 256, 0, st>>>(g);
    if (g.rgbmax < INFINITY) k_gchain_sym<true><<<grid, kGT, 0, st>>>(g);
    else k_gchain_sym<false><<<grid, kGT, 0, st>>>(g);
    k_gfin_out<<<ba, 256, 0, st>>>(g);
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
