// Symmetric (Newton's third law) kernels of the differentiable GB energy:
// every unordered pair of a replica is evaluated once and contributes to both
// atoms, with the decomposition of the engine's FP32 passes -- a CTA of 128
// threads owns a 256-atom i-tile (two atoms per lane) and sweeps 32-atom
// j-tiles of the upper triangle in groups of four staged by all threads;
// partner-side partials rotate across lanes by warp shuffle and land, like the
// i-side ones, in int64 fixed-point accumulators (exact, order independent).
// Work items are decoded from the block index (replica, i-tile, chunk of
// j-tiles); chunks past the end of a row exit at once.  Nothing is allocated:
// accumulators live in the caller's workspace.
//
// Far pairs: a bound kernel takes s_max and rt_max over every replica's atoms;
// for r >= r_far = max(s_max / 0.35, s_max + rt_max) every descreening
// integral of the pair, and its r-, rt- and s-derivatives, are in the
// disjoint-sphere series regime (dH/drt = 0 there).
#pragma once
#include "cph_device.cuh"

namespace cph {
namespace grad {

constexpr int kGT = 128;     // threads per CTA
constexpr int kGI = 256;     // atoms per i-tile
constexpr int kGJ = 32;      // atoms per j-tile
constexpr int kGG = 4;       // j-tiles staged per barrier
constexpr int kGChunk = 16;  // j-tiles per work item
constexpr float kFar = 1.0e4f; // padding / invalid atoms sit this far away

struct SView {
    int n_rep, n, n_itile, n_jtile, n_chunk;
    const float *x, *q, *rho, *screen;
    double tau, sqrt_k, alpha, beta, gamma, offset;
    // per replica-atom (index r * n + a); int64 slots alias double slots that
    // are not live at the same time (see ws_carve_sym)
    double *psi, *R, *dEdR, *c, *dq, *gpsi;
    long long *Hfix, *dRfix, *dqfix, *gfix, *artfix, *asfix;
    long long* eacc;      // [n_rep] energies, fixed point 2^32
    unsigned int* bound;  // [2]: float bits of s_max, rt_max
    double* E;
    const double* dE;
    float *dx, *dqo, *drho;
};

// max over every replica's atoms of s = screen (rho - offset) and rt = rho - offset
__global__ void k_gbound(SView g) {
    const size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= (size_t)g.n_rep * g.n) return;
    const float rt = g.rho[a] - (float)g.offset;
    const float s = g.screen[a % g.n] * rt;
    // positive floats order like their bit patterns
    atomicMax(&g.bound[0], __float_as_uint(fmaxf(s, 0.f)));
    atomicMax(&g.bound[1], __float_as_uint(fmaxf(rt, 0.f)));
}

__device__ __forceinline__ float gfar2(const SView& g) {
    const float smax = __uint_as_float(g.bound[0]), rtmax = __uint_as_float(g.bound[1]);
    const float rf = fmaxf(smax / kHctXmax, smax + rtmax) * 1.0001f;
    return rf * rf;
}

struct GItem {
    int rep, i0, jt0, jt1;
    bool ok;
};

__device__ __forceinline__ GItem gitem(const SView& g) {
    GItem it;
    const int per_rep = g.n_itile * g.n_chunk;
    it.rep = blockIdx.x / per_rep;
    const int rem = blockIdx.x % per_rep;
    const int ti = rem / g.n_chunk, ch = rem % g.n_chunk;
    it.i0 = ti * kGI;
    it.jt0 = (it.i0 / kGJ) + ch * kGChunk;
    it.jt1 = min(g.n_jtile, it.jt0 + kGChunk);
    it.ok = it.jt0 < g.n_jtile;
    return it;
}

// skip mask of one i atom for the j-tile at j0: partners j <= i or j >= n
__device__ __forceinline__ uint32_t gskip(int i, bool vi, int j0, int n) {
    if (!vi) return 0xffffffffu;
    uint32_t skip = 0u;
    const int d = i - j0;
    if (d >= 31) skip = 0xffffffffu;
    else if (d >= 0) skip = (2u << d) - 1u;
    const int nv = n - j0;
    if (nv < 32) skip |= ~((nv <= 0) ? 0u : (0xffffffffu >> (32 - nv)));
    return skip;
}

__device__ __forceinline__ bool gmasked(int jt, int i0, int n) {
    // j-tiles meeting the i-tile's own atoms, and the ragged last tile
    return (jt * kGJ < i0 + kGI) || ((jt + 1) * kGJ > n);
}

// ------------------------------------------------------------ Born radii
__global__ void __launch_bounds__(kGT, 8) k_gborn_sym(SView g) {
    __shared__ float4 sa[kGG * kGJ];
    __shared__ float2 sb[kGG * kGJ];
    __shared__ float red[kGG][4][kGJ];
    const GItem it = gitem(g);
    if (!it.ok) return;
    const int n = g.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* X = g.x + (size_t)it.rep * n * 3;
    const float* RH = g.rho + (size_t)it.rep * n;
    const size_t base = (size_t)it.rep * n;
    const float off = (float)g.offset, rfar2 = gfar2(g);
    const float cx = X[3 * it.i0], cy = X[3 * it.i0 + 1], cz = X[3 * it.i0 + 2];
    int ii[2];
    bool vi[2];
    float xi[2], yi[2], zi[2], si[2], rti[2], irti[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < n;
        const int i = vi[u] ? ii[u] : it.i0;
        xi[u] = vi[u] ? X[3 * i] - cx : -kFar;
        yi[u] = vi[u] ? X[3 * i + 1] - cy : -kFar;
        zi[u] = vi[u] ? X[3 * i + 2] - cz : -kFar;
        rti[u] = vi[u] ? RH[i] - off : 1.f;
        si[u] = vi[u] ? g.screen[i] * rti[u] : 0.f;
        irti[u] = 1.f / rti[u];
    }
    long long hx[2] = {0, 0};
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kGG) {
        const int ng = min(kGG, it.jt1 - g0);
        __syncthreads();
        if (tid < ng * kGJ) {
            const int j = g0 * kGJ + tid;
            if (j < n) {
                const float rtj = RH[j] - off;
                sa[tid] = make_float4(X[3 * j] - cx, X[3 * j + 1] - cy, X[3 * j + 2] - cz, rtj);
                sb[tid] = make_float2(g.screen[j] * rtj, 1.f / rtj);
            } else {
                sa[tid] = make_float4(kFar, kFar, kFar, 1.f);
                sb[tid] = make_float2(0.f, 1.f);
            }
        }
        __syncthreads();
        for (int gt = 0; gt < ng; ++gt) {
            const int jt = g0 + gt, j0 = jt * kGJ;
            const bool msk = gmasked(jt, it.i0, n);
            uint32_t skip[2] = {0u, 0u};
            if (msk) {
                skip[0] = gskip(ii[0], vi[0], j0, n);
                skip[1] = gskip(ii[1], vi[1], j0, n);
            }
            const float4* A4 = sa + gt * kGJ;
            const float2* B2 = sb + gt * kGJ;
            float ah[2] = {0.f, 0.f}, jh = 0.f;
#pragma unroll 2
            for (int k = 0; k < kGJ; ++k) {
                const int jj = (lane + k) & (kGJ - 1);
                const float4 A = A4[jj];
                const float2 B = B2[jj];
                float r2[2], rinv[2], hi[2], hj[2];
                bool sk[2], nr[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float dx = xi[u] - A.x, dy = yi[u] - A.y, dz = zi[u] - A.z;
                    r2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    sk[u] = msk && ((skip[u] >> jj) & 1u);
                    r2[u] = sk[u] ? 1.f : r2[u];
                    rinv[u] = rsqrt_ftz(r2[u]);
                    const float x1 = B.x * rinv[u], x2 = si[u] * rinv[u];
                    hi[u] = x1 * x1 * x1 * hct_series_h(x1 * x1) * rinv[u];
                    hj[u] = x2 * x2 * x2 * hct_series_h(x2 * x2) * rinv[u];
                    nr[u] = r2[u] < rfar2;
                }
                if (__any_sync(0xffffffffu, nr[0] || nr[1])) {
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        if (nr[u]) {
                            const float r = r2[u] * rinv[u];
                            hi[u] = hct(r, rinv[u], rti[u], irti[u], B.x);
                            hj[u] = hct(r, rinv[u], A.w, B.y, si[u]);
                        }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    ah[u] += sk[u] ? 0.f : hi[u];
                    jh += sk[u] ? 0.f : hj[u];
                }
                jh = __shfl_sync(0xffffffffu, jh, (lane + 1) & 31);
            }
            hx[0] += to_fixed(ah[0], (float)kScaleH);
            hx[1] += to_fixed(ah[1], (float)kScaleH);
            red[gt][warp][lane] = jh;
        }
        __syncthreads();
        if (tid < ng * kGJ) {
            const int gt = tid / kGJ, j = tid % kGJ;
            const float v = red[gt][0][j] + red[gt][1][j] + red[gt][2][j] + red[gt][3][j];
            const int jg = g0 * kGJ + tid;
            if (jg < n) atomicAdd((unsigned long long*)&g.Hfix[base + jg], (unsigned long long)to_fixed(v, (float)kScaleH));
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (vi[u]) atomicAdd((unsigned long long*)&g.Hfix[base + ii[u]], (unsigned long long)hx[u]);
}

// psi, R (FP64); resets the fixed-point accumulators of the pair passes.
// Hfix and dRfix share a slot: H is read, then the slot starts dE/dR at zero.
__global__ void k_gfin_born(SView g) {
    const size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= (size_t)g.n_rep * g.n) return;
    const double rho = g.rho[a], rt = rho - g.offset;
    const double psi = 0.5 * rt * ((double)g.Hfix[a] / kScaleH);
    const double th = tanh(psi * (g.alpha + psi * (-g.beta + psi * g.gamma)));
    const double R = 1.0 / (1.0 / rt - th / rho);
    g.psi[a] = psi;
    g.R[a] = R;
    g.gpsi[a] = R * R * (1.0 - th * th) * (g.alpha + psi * (-2.0 * g.beta + 3.0 * g.gamma * psi)) / rho; // dR/dpsi for now
    g.dRfix[a] = 0; // same slot as Hfix
    g.dqfix[a] = 0;
    g.gfix[3 * a] = 0;
    g.gfix[3 * a + 1] = 0;
    g.gfix[3 * a + 2] = 0;
    if (a % g.n == 0) g.eacc[a / g.n] = 0;
}

// ------------------------------------------------------------ GB pair pass
// Per unordered pair (qs = sqrt(k) q): E += qs_i qs_j / f (times -tau at the
// end); dE/dR both ways; sum_j qs_j / f for dE/dq both ways; the direct
// gradient tau qq (1 - e/4) / f^3 (x_i - x_j) to i and its negative to j.
template <bool BACKWARD>
__global__ void __launch_bounds__(kGT, 6) k_gpair_sym(SView g) {
    __shared__ float4 sa[kGG * kGJ], sb[kGG * kGJ];
    __shared__ float red[kGG][4][kGJ][5];
    __shared__ long long sfx[kGI][5];
    __shared__ double ered[kGT / 32];
    const GItem it = gitem(g);
    if (!it.ok) return;
    const int n = g.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* X = g.x + (size_t)it.rep * n * 3;
    const float* Q = g.q + (size_t)it.rep * n;
    const size_t base = (size_t)it.rep * n;
    const float sqk = (float)g.sqrt_k, tau = (float)g.tau;
    const float cx = X[3 * it.i0], cy = X[3 * it.i0 + 1], cz = X[3 * it.i0 + 2];
    int ii[2];
    bool vi[2];
    float xi[2], yi[2], zi[2], qi[2], Ri[2], dki[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < n;
        const int i = vi[u] ? ii[u] : it.i0;
        xi[u] = vi[u] ? X[3 * i] - cx : -kFar;
        yi[u] = vi[u] ? X[3 * i + 1] - cy : -kFar;
        zi[u] = vi[u] ? X[3 * i + 2] - cz : -kFar;
        qi[u] = vi[u] ? Q[i] * sqk : 0.f;
        Ri[u] = vi[u] ? (float)g.R[base + i] : 1.f;
        dki[u] = vi[u] ? (float)(0.25 * 1.4426950408889634 / g.R[base + i]) : 1.f;
#pragma unroll
        for (int c = 0; c < 5; ++c) sfx[warp * 64 + u * 32 + lane][c] = 0;
    }
    KSum<float> egb;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kGG) {
        const int ng = min(kGG, it.jt1 - g0);
        __syncthreads();
        if (tid < ng * kGJ) {
            const int j = g0 * kGJ + tid;
            if (j < n) {
                sa[tid] = make_float4(X[3 * j] - cx, X[3 * j + 1] - cy, X[3 * j + 2] - cz, Q[j] * sqk);
                sb[tid] = make_float4((float)g.R[base + j], (float)(1.0 / g.R[base + j]), 0.f, 0.f);
            } else {
                sa[tid] = make_float4(kFar, kFar, kFar, 0.f);
                sb[tid] = make_float4(1.f, 1.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        for (int gt = 0; gt < ng; ++gt) {
            const int jt = g0 + gt, j0 = jt * kGJ;
            const bool msk = gmasked(jt, it.i0, n);
            uint32_t skip[2] = {0u, 0u};
            if (msk) {
                skip[0] = gskip(ii[0], vi[0], j0, n);
                skip[1] = gskip(ii[1], vi[1], j0, n);
            }
            const float4* A4 = sa + gt * kGJ;
            const float4* B4 = sb + gt * kGJ;
            float ai[2][5] = {{0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f}};
            float aj[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
            for (int k = 0; k < kGJ; ++k) {
                const int jj = (lane + k) & (kGJ - 1);
                const float4 A = A4[jj];
                const float4 B = B4[jj];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float dx = xi[u] - A.x, dy = yi[u] - A.y, dz = zi[u] - A.z;
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const bool sk = msk && ((skip[u] >> jj) & 1u);
                    r2 = sk ? 1.f : r2;
                    const float m = sk ? 0.f : 1.f;
                    const float D2 = r2 * (dki[u] * B.y);
                    const float e = exp2_ftz(-D2);
                    const float fi = m * rsqrt_ftz(fmaf(Ri[u] * B.x, e, r2));
                    const float qq = qi[u] * A.w;
                    egb.add(qq * fi);
                    if (BACKWARD) {
                        const float qf3 = qq * fi * fi * fi;
                        const float t = qf3 * e * fmaf(D2, kLn2, 1.f);
                        ai[u][0] = fmaf(t, B.x, ai[u][0]);
                        aj[0] = fmaf(t, Ri[u], aj[0]);
                        ai[u][1] = fmaf(A.w, fi, ai[u][1]);
                        aj[1] = fmaf(qi[u], fi, aj[1]);
                        const float gt2 = tau * qf3 * fmaf(-0.25f, e, 1.f);
                        ai[u][2] = fmaf(gt2, dx, ai[u][2]);
                        ai[u][3] = fmaf(gt2, dy, ai[u][3]);
                        ai[u][4] = fmaf(gt2, dz, ai[u][4]);
                        aj[2] = fmaf(-gt2, dx, aj[2]);
                        aj[3] = fmaf(-gt2, dy, aj[3]);
                        aj[4] = fmaf(-gt2, dz, aj[4]);
                    }
                }
                if (BACKWARD) {
                    const int src = (lane + 1) & 31;
#pragma unroll
                    for (int c = 0; c < 5; ++c) aj[c] = __shfl_sync(0xffffffffu, aj[c], src);
                }
            }
            if (BACKWARD) {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    long long* row = sfx[warp * 64 + u * 32 + lane];
#pragma unroll
                    for (int c = 0; c < 5; ++c) row[c] += to_fixed(ai[u][c], (float)kScaleE);
                }
#pragma unroll
                for (int c = 0; c < 5; ++c) red[gt][warp][lane][c] = aj[c];
            }
        }
        if (BACKWARD) {
            __syncthreads();
            for (int v = tid; v < ng * kGJ * 5; v += kGT) {
                const int gt = v / (kGJ * 5), rem = v % (kGJ * 5), j = rem / 5, c = rem % 5;
                const float sum = red[gt][0][j][c] + red[gt][1][j][c] + red[gt][2][j][c] + red[gt][3][j][c];
                const int jg = (g0 + gt) * kGJ + j;
                if (jg < n) {
                    long long* dst = c == 0 ? &g.dRfix[base + jg]
                                   : (c == 1 ? &g.dqfix[base + jg] : &g.gfix[3 * (base + jg) + (c - 2)]);
                    atomicAdd((unsigned long long*)dst, (unsigned long long)to_fixed(sum, (float)kScaleE));
                }
            }
        }
    }
    if (BACKWARD) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!vi[u]) continue;
            const long long* row = sfx[warp * 64 + u * 32 + lane];
            const size_t a = base + ii[u];
            atomicAdd((unsigned long long*)&g.dRfix[a], (unsigned long long)row[0]);
            atomicAdd((unsigned long long*)&g.dqfix[a], (unsigned long long)row[1]);
            atomicAdd((unsigned long long*)&g.gfix[3 * a], (unsigned long long)row[2]);
            atomicAdd((unsigned long long*)&g.gfix[3 * a + 1], (unsigned long long)row[3]);
            atomicAdd((unsigned long long*)&g.gfix[3 * a + 2], (unsigned long long)row[4]);
        }
    }
    // pair energy of this item: compensated lane sums, FP64 block reduction
    double e0 = (double)egb.s - (double)egb.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e0 += __shfl_down_sync(0xffffffffu, e0, o);
    if (lane == 0) ered[warp] = e0;
    __syncthreads();
    if (tid == 0) {
        const double v = ered[0] + ered[1] + ered[2] + ered[3];
        atomicAdd((unsigned long long*)&g.eacc[it.rep], (unsigned long long)__double2ll_rn(-g.tau * v * kScaleE));
    }
}

// self energy; for the backward also dE/dR, c = dE/dR dR/dpsi rt/2, dE/dq
template <bool BACKWARD>
__global__ void k_gfin_c(SView g) {
    const size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= (size_t)g.n_rep * g.n) return;
    const double q = (double)g.q[a] * g.sqrt_k, R = g.R[a];
    atomicAdd((unsigned long long*)&g.eacc[a / g.n], (unsigned long long)__double2ll_rn(-0.5 * g.tau * q * q / R * kScaleE));
    if (!BACKWARD) return;
    const double dEdR = 0.5 * g.tau * ((double)g.dRfix[a] / kScaleE + q * q / (R * R));
    const double rt = (double)g.rho[a] - g.offset;
    const double gpsi = dEdR * g.gpsi[a]; // gpsi slot held dR/dpsi
    const double dq = -g.tau * g.sqrt_k * ((double)g.dqfix[a] / kScaleE + q / R);
    g.dEdR[a] = dEdR; // same slot as dRfix
    g.gpsi[a] = gpsi;
    g.c[a] = gpsi * 0.5 * rt;
    g.dq[a] = dq; // same slot as dqfix
    g.artfix[a] = 0;
    g.asfix[a] = 0;
}

__global__ void k_genergy_out(SView g) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < g.n_rep) g.E[r] = (double)g.eacc[r] / kScaleE;
}

// ------------------------------------------------- chain-rule adjoint pass
// Per unordered pair, with c = dE/dpsi rt/2 of each atom:
//   gradient  (c_i dH(r; rt_i, s_j)/dr + c_j dH(r; rt_j, s_i)/dr) (x_i - x_j)/r to i, minus to j;
//   art_i += dH(r; rt_i, s_j)/drt,   as_i += c_j dH(r; rt_j, s_i)/ds   (and i <-> j),
// which k_gfin_out turns into dE/drho.
__device__ __forceinline__ float hct_dr_series(float rinv2, float rinv, float s) {
    const float x = s * rinv, y = x * x;
    return -x * y * hct_series_dr(y) * rinv2;
}

__device__ __forceinline__ float ds_series(float rinv2, float rinv, float s) {
    const float x = s * rinv, y = x * x;
    return y * hct_series_ds(y) * rinv2;
}

__global__ void __launch_bounds__(kGT, 6) k_gchain_sym(SView g) {
    __shared__ float4 sa[kGG * kGJ], sb[kGG * kGJ];
    __shared__ float red[kGG][4][kGJ][5];
    __shared__ long long sfx[kGI][5];
    const GItem it = gitem(g);
    if (!it.ok) return;
    const int n = g.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* X = g.x + (size_t)it.rep * n * 3;
    const float* RH = g.rho + (size_t)it.rep * n;
    const size_t base = (size_t)it.rep * n;
    const float off = (float)g.offset, rfar2 = gfar2(g);
    const float cx = X[3 * it.i0], cy = X[3 * it.i0 + 1], cz = X[3 * it.i0 + 2];
    int ii[2];
    bool vi[2];
    float xi[2], yi[2], zi[2], ci[2], si[2], rti[2], irti[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < n;
        const int i = vi[u] ? ii[u] : it.i0;
        xi[u] = vi[u] ? X[3 * i] - cx : -kFar;
        yi[u] = vi[u] ? X[3 * i + 1] - cy : -kFar;
        zi[u] = vi[u] ? X[3 * i + 2] - cz : -kFar;
        ci[u] = vi[u] ? (float)g.c[base + i] : 0.f;
        rti[u] = vi[u] ? RH[i] - off : 1.f;
        si[u] = vi[u] ? g.screen[i] * rti[u] : 0.f;
        irti[u] = 1.f / rti[u];
#pragma unroll
        for (int c = 0; c < 5; ++c) sfx[warp * 64 + u * 32 + lane][c] = 0;
    }
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kGG) {
        const int ng = min(kGG, it.jt1 - g0);
        __syncthreads();
        if (tid < ng * kGJ) {
            const int j = g0 * kGJ + tid;
            if (j < n) {
                const float rtj = RH[j] - off;
                sa[tid] = make_float4(X[3 * j] - cx, X[3 * j + 1] - cy, X[3 * j + 2] - cz, (float)g.c[base + j]);
                sb[tid] = make_float4(g.screen[j] * rtj, rtj, 1.f / rtj, 0.f);
            } else {
                sa[tid] = make_float4(kFar, kFar, kFar, 0.f);
                sb[tid] = make_float4(0.f, 1.f, 1.f, 0.f);
            }
        }
        __syncthreads();
        for (int gt = 0; gt < ng; ++gt) {
            const int jt = g0 + gt, j0 = jt * kGJ;
            const bool msk = gmasked(jt, it.i0, n);
            uint32_t skip[2] = {0u, 0u};
            if (msk) {
                skip[0] = gskip(ii[0], vi[0], j0, n);
                skip[1] = gskip(ii[1], vi[1], j0, n);
            }
            const float4* A4 = sa + gt * kGJ;
            const float4* B4 = sb + gt * kGJ;
            float ai[2][5] = {{0.f, 0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f, 0.f}};
            float aj[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
            for (int k = 0; k < kGJ; ++k) {
                const int jj = (lane + k) & (kGJ - 1);
                const float4 A = A4[jj];
                const float4 B = B4[jj];
                float dx[2], dy[2], dz[2], r2[2], rinv[2], hri[2], hrj[2], hti[2], htj[2], hsi[2], hsj[2];
                bool sk[2], nr[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    dx[u] = xi[u] - A.x;
                    dy[u] = yi[u] - A.y;
                    dz[u] = zi[u] - A.z;
                    r2[u] = fmaf(dx[u], dx[u], fmaf(dy[u], dy[u], dz[u] * dz[u]));
                    sk[u] = msk && ((skip[u] >> jj) & 1u);
                    r2[u] = sk[u] ? 1.f : r2[u];
                    rinv[u] = rsqrt_ftz(r2[u]);
                    const float rinv2 = rinv[u] * rinv[u];
                    hri[u] = hct_dr_series(rinv2, rinv[u], B.x);
                    hrj[u] = hct_dr_series(rinv2, rinv[u], si[u]);
                    hsi[u] = ds_series(rinv2, rinv[u], si[u]); // dH(r; rt_j, s_i)/ds
                    hsj[u] = ds_series(rinv2, rinv[u], B.x);   // dH(r; rt_i, s_j)/ds
                    hti[u] = 0.f;
                    htj[u] = 0.f;
                    nr[u] = r2[u] < rfar2;
                }
                if (__any_sync(0xffffffffu, nr[0] || nr[1])) {
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        if (nr[u]) {
                            const float r = r2[u] * rinv[u];
                            hri[u] = hct_dr(r, rinv[u], rti[u], B.x);
                            hrj[u] = hct_dr(r, rinv[u], B.y, si[u]);
                            hsi[u] = hct_ds(r, rinv[u], B.y, si[u]);
                            hsj[u] = hct_ds(r, rinv[u], rti[u], B.x);
                            hti[u] = hct_drt(r, rti[u], irti[u], B.x);
                            htj[u] = hct_drt(r, B.y, B.z, si[u]);
                        }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const float m = sk[u] ? 0.f : 1.f;
                    const float t = m * (ci[u] * hri[u] + A.w * hrj[u]) * rinv[u];
                    ai[u][0] = fmaf(t, dx[u], ai[u][0]);
                    ai[u][1] = fmaf(t, dy[u], ai[u][1]);
                    ai[u][2] = fmaf(t, dz[u], ai[u][2]);
                    aj[0] = fmaf(-t, dx[u], aj[0]);
                    aj[1] = fmaf(-t, dy[u], aj[1]);
                    aj[2] = fmaf(-t, dz[u], aj[2]);
                    ai[u][3] = fmaf(m, hti[u], ai[u][3]);
                    aj[3] = fmaf(m, htj[u], aj[3]);
                    ai[u][4] = fmaf(m * A.w, hsi[u], ai[u][4]);
                    aj[4] = fmaf(m * ci[u], hsj[u], aj[4]);
                }
                const int src = (lane + 1) & 31;
#pragma unroll
                for (int c = 0; c < 5; ++c) aj[c] = __shfl_sync(0xffffffffu, aj[c], src);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                long long* row = sfx[warp * 64 + u * 32 + lane];
#pragma unroll
                for (int c = 0; c < 5; ++c) row[c] += to_fixed(ai[u][c], (float)kScaleE);
            }
#pragma unroll
            for (int c = 0; c < 5; ++c) red[gt][warp][lane][c] = aj[c];
        }
        __syncthreads();
        for (int v = tid; v < ng * kGJ * 5; v += kGT) {
            const int gt = v / (kGJ * 5), rem = v % (kGJ * 5), j = rem / 5, c = rem % 5;
            const float sum = red[gt][0][j][c] + red[gt][1][j][c] + red[gt][2][j][c] + red[gt][3][j][c];
            const int jg = (g0 + gt) * kGJ + j;
            if (jg < n) {
                long long* dst = c < 3 ? &g.gfix[3 * (base + jg) + c] : (c == 3 ? &g.artfix[base + jg] : &g.asfix[base + jg]);
                atomicAdd((unsigned long long*)dst, (unsigned long long)to_fixed(sum, (float)kScaleE));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (!vi[u]) continue;
        const long long* row = sfx[warp * 64 + u * 32 + lane];
        const size_t a = base + ii[u];
        atomicAdd((unsigned long long*)&g.gfix[3 * a], (unsigned long long)row[0]);
        atomicAdd((unsigned long long*)&g.gfix[3 * a + 1], (unsigned long long)row[1]);
        atomicAdd((unsigned long long*)&g.gfix[3 * a + 2], (unsigned long long)row[2]);
        atomicAdd((unsigned long long*)&g.artfix[a], (unsigned long long)row[3]);
        atomicAdd((unsigned long long*)&g.asfix[a], (unsigned long long)row[4]);
    }
}

// outputs: dx, dq, drho scaled by the upstream gradient of the replica
__global__ void k_gfin_out(SView g) {
    const size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= (size_t)g.n_rep * g.n) return;
    const int r = (int)(a / g.n);
    const double up = g.dE[r];
    const double rho = g.rho[a], rt = rho - g.offset, R = g.R[a], psi = g.psi[a];
    const double th = tanh(psi * (g.alpha + psi * (-g.beta + psi * g.gamma)));
    const double dr = g.dEdR[a] * R * R * (1.0 / (rt * rt) - th / (rho * rho)) + g.gpsi[a] * psi / rt +
                      g.c[a] * ((double)g.artfix[a] / kScaleE) +
                      (double)g.screen[a % g.n] * ((double)g.asfix[a] / kScaleE);
    g.dx[3 * a] = (float)(up * ((double)g.gfix[3 * a] / kScaleE));
    g.dx[3 * a + 1] = (float)(up * ((double)g.gfix[3 * a + 1] / kScaleE));
    g.dx[3 * a + 2] = (float)(up * ((double)g.gfix[3 * a + 2] / kScaleE));
    g.dqo[a] = (float)(up * g.dq[a]);
    g.drho[a] = (float)(up * dr);
}

} // namespace grad
} // namespace cph
