// Symmetric (Newton's third law) kernels of the differentiable GB energy:
// every unordered pair of a replica is evaluated once and contributes to both
// atoms, with the decomposition of the engine's FP32 passes -- a CTA of 128
// threads owns a 256-atom i-tile (two atoms per lane) and sweeps 32-atom
// j-tiles of the upper triangle two at a time (tile pairs, packed f32x2
// arithmetic, see cph_pair_tiles.cuh), eight tiles staged per barrier;
// partner-side partials rotate across lanes by warp shuffle and land, like the
// i-side ones, in int64 fixed-point accumulators (exact, order independent).
// Coordinates are used as given (x_i - x_j is one FP32 rounding).
// Work items are decoded from the block index (replica, i-tile, chunk of
// j-tiles); chunks past the end of a row exit at once.  Nothing is allocated:
// accumulators live in the caller's workspace.
//
// Far pairs: a bound kernel takes s_max and rt_max over every replica's atoms;
// for r >= r_far = max(s_max / 0.35, s_max + rt_max) every descreening
// integral of the pair, and its r-, rt- and s-derivatives, are in the
// disjoint-sphere series regime (dH/drt = 0 there).  A Born-radius cutoff rc
// adds the band rc - s_max < r < rc + s_max to the closed forms and zeroes
// every pair beyond it (see PairBand).
#pragma once
#include "cph_device.cuh"
#include "cph_pair_tiles.cuh"

namespace cph {
namespace grad {

constexpr int kGT = 128;     // threads per CTA
constexpr int kGI = 256;     // atoms per i-tile
constexpr int kGJ = kTileJ;   // atoms per j-tile
constexpr int kGG = 8;       // j-tiles staged per barrier (four tile pairs)
constexpr int kGChunk = 16;  // j-tiles per work item
constexpr float kFar = 1.0e4f; // padding / invalid atoms sit this far away

struct SView {
    int n_rep, n, n_itile, n_jtile, n_chunk;
    const float *x, *q, *rho, *screen;
    double tau, sqrt_k, alpha, beta, gamma, offset;
    // Debye-Hueckel salt screening: kappa (1/A), 1/eps_in, 1/eps_out; tau_pair is
    // the factor the finishing kernels apply to the pair sums (tau without
    // salt; 1 with salt, whose pair terms carry tau(f) per pair)
    double kappa, inv_eps_in, inv_eps_out, tau_pair;
    // FP32 copies for the pair kernels, rounded once on the host (a reload
    // under register pressure then reads a parameter instead of converting
    // the double again on the narrow FP64 pipe)
    float tau32, sqk32, iei32, ieo32, kap32, off32, rgbmax32;
    double sa_gamma, sa_probe; // nonpolar surface term (ACE), 0 = off
    double rgbmax;             // Born-radius cutoff, INFINITY = none
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
    const float rt = g.rho[a] - g.off32;
    const float s = g.screen[a % g.n] * rt;
    // positive floats order like their bit patterns
    atomicMax(&g.bound[0], __float_as_uint(fmaxf(s, 0.f)));
    atomicMax(&g.bound[1], __float_as_uint(fmaxf(rt, 0.f)));
}

__device__ __forceinline__ PairBand gband(const SView& g) {
    const float smax = __uint_as_float(g.bound[0]), rtmax = __uint_as_float(g.bound[1]);
    const float rf = fmaxf(smax / kHctXmax, smax + rtmax) * 1.0001f;
    return pair_band(rf * rf, smax, g.rgbmax32);
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
template <bool CUT>
__global__ void __launch_bounds__(kGT, 6) k_gborn_sym(SView g) {
    __shared__ BoJs sj[kGG / 2];
    __shared__ float red[kGG][4][kGJ];
    const GItem it = gitem(g);
    if (!it.ok) return;
    const int n = g.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* X = g.x + (size_t)it.rep * n * 3;
    const float* RH = g.rho + (size_t)it.rep * n;
    const size_t base = (size_t)it.rep * n;
    const float off = g.off32;
    const PairBand band = gband(g);
    int ii[2];
    bool vi[2];
    BoI2 I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < n;
        const int i = vi[u] ? ii[u] : it.i0;
        const float rt = vi[u] ? RH[i] - off : 1.f, si = vi[u] ? g.screen[i] * rt : 0.f;
        I[u].x = splat<float2>(vi[u] ? X[3 * i] : -kFar);
        I[u].y = splat<float2>(vi[u] ? X[3 * i + 1] : -kFar);
        I[u].z = splat<float2>(vi[u] ? X[3 * i + 2] : -kFar);
        I[u].s2 = splat<float2>(si * si);
        I[u].s3 = splat<float2>(si * si * si);
        I[u].s = si;
        I[u].rt = rt;
        I[u].irt = 1.f / rt;
    }
    long long hx[2] = {0, 0};
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kGG) {
        const int ng = min(kGG, it.jt1 - g0), npair = (ng + 1) >> 1;
        __syncthreads();
        // stage the tile pairs: thread (pair, copy, entry) writes whole rows
        for (int q = tid; q < npair * 2 * kGJ; q += kGT) {
            const int pr = q >> 6, cpy = (q >> 5) & 1, e = q & 31;
            float v[2][6];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gt = 2 * pr + h, j = (g0 + gt) * kGJ + e;
                if (gt < ng && j < n) {
                    const float rt = RH[j] - off;
                    v[h][0] = -X[3 * j]; v[h][1] = -X[3 * j + 1]; v[h][2] = -X[3 * j + 2];
                    v[h][3] = g.screen[j] * rt; v[h][4] = rt; v[h][5] = 1.f / rt;
                } else { // padding: far away, no sphere
                    v[h][0] = kFar; v[h][1] = kFar; v[h][2] = kFar;
                    v[h][3] = 0.f; v[h][4] = 1.f; v[h][5] = 1.f;
                }
            }
            BoJs& S = sj[pr];
            const int r = e + cpy * kGJ;
            const float s2a = v[0][3] * v[0][3], s2b = v[1][3] * v[1][3];
            S.a[r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
            S.b[r] = make_float4(v[0][2], v[1][2], s2a, s2b);
            S.c[r] = make_float4(s2a * v[0][3], s2b * v[1][3], v[0][3], v[1][3]);
            S.n[r] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
        }
        __syncthreads();
        for (int pr = 0; pr < npair; ++pr) {
            float2 jh = make_float2(0.f, 0.f);
            float2 ah[2] = {{0.f, 0.f}, {0.f, 0.f}};
            uint32_t sk[2][2] = {{0u, 0u}, {0u, 0u}};
            bool masked = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jt = g0 + 2 * pr + h;
                if (jt < it.jt1 && gmasked(jt, it.i0, n)) {
                    masked = true;
#pragma unroll
                    for (int u = 0; u < 2; ++u) sk[u][h] = gskip(ii[u], vi[u], jt * kGJ, n);
                }
            }
            if (masked) born_tile<true, CUT>(sj[pr], lane, I, ah, jh, sk, band);
            else born_tile<false, CUT>(sj[pr], lane, I, ah, jh, sk, band);
#pragma unroll
            for (int u = 0; u < 2; ++u)
                hx[u] += to_fixed(ah[u].x, (float)kScaleH) + to_fixed(ah[u].y, (float)kScaleH);
            red[2 * pr][warp][lane] = jh.x;
            red[2 * pr + 1][warp][lane] = jh.y;
        }
        __syncthreads();
        for (int q = tid; q < ng * kGJ; q += kGT) {
            const int gt = q / kGJ, j = q % kGJ;
            const float v = red[gt][0][j] + red[gt][1][j] + red[gt][2][j] + red[gt][3][j];
            const int jg = g0 * kGJ + q;
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
    const double rho = g.rho[a], rt = rho - g.offset, irho = 1.0 / rho;
    const double psi = 0.5 * rt * ((double)g.Hfix[a] / kScaleH);
    const double th = tanh(psi * (g.alpha + psi * (-g.beta + psi * g.gamma)));
    const double R = 1.0 / (1.0 / rt - th * irho);
    g.psi[a] = psi;
    g.R[a] = R;
    g.gpsi[a] = R * R * (1.0 - th * th) * (g.alpha + psi * (-2.0 * g.beta + 3.0 * g.gamma * psi)) * irho; // dR/dpsi for now
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
// Packed over partner tiles (A, B) like the engine's passes.
struct GpI2 {
    float2 x, y, z, q, R, dk; // the i atom's value in both halves
};

struct GpJs {
    float4 a[2 * kGJ]; // (-xA, -xB, -yA, -yB)
    float4 b[2 * kGJ]; // (-zA, -zB, qA, qB)
    float4 c[2 * kGJ]; // (RA, RB, 1/RA, 1/RB)
};

// SALT: every GB pair term carries tau(f) = 1/eps_in - exp(-kappa f)/eps_out
// (energy, dE/dq) and taud(f) = tau(f) - kappa f exp(-kappa f)/eps_out (dE/df),
// f the effective distance; the finishing kernels then scale the pair sums by
// 1 instead of tau.  Salt steps always take the full form.
template <bool MASKED, bool BACKWARD, bool SALT>
__device__ __forceinline__ void gpair_tile(const GpJs& sj, int lane, const GpI2 (&I)[2], float2 (&ai)[2][5],
                                           float2 (&aj)[5], float2 (&ei)[2], const uint32_t (&sk)[2][2],
                                           float tau, float iei, float ieo, float kappa) {
    const int src = (lane + 1) & 31;
    const float2 ln2 = splat<float2>(kLn2), one = splat<float2>(1.f), tau2 = splat<float2>(tau),
                 mtau4 = splat<float2>(-0.25f * tau), ie = splat<float2>(iei), ieo2 = splat<float2>(ieo),
                 mone = splat<float2>(-1.f), q25 = splat<float2>(0.25f), kap2 = splat<float2>(kappa);
    const float kl = kappa * kLog2e;
#pragma unroll 2
    for (int k = 0; k < kGJ; ++k) {
        const float4 A = sj.a[lane + k], B = sj.b[lane + k], C = sj.c[lane + k];
        const float2 qj = make_float2(B.z, B.w), Rj = make_float2(C.x, C.y);
        float2 dx[2], dy[2], dz[2], r2[2], D2[2];
        bool s0[2] = {false, false}, s1[2] = {false, false};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            dx[u] = __fadd2_rn(I[u].x, make_float2(A.x, A.y));
            dy[u] = __fadd2_rn(I[u].y, make_float2(A.z, A.w));
            dz[u] = __fadd2_rn(I[u].z, make_float2(B.x, B.y));
            r2[u] = __ffma2_rn(dx[u], dx[u], __ffma2_rn(dy[u], dy[u], __fmul2_rn(dz[u], dz[u])));
            if (MASKED) {
                const int jj = (lane + k) & (kGJ - 1);
                s0[u] = (sk[u][0] >> jj) & 1u;
                s1[u] = (sk[u][1] >> jj) & 1u;
                r2[u].x = s0[u] ? 1.f : r2[u].x;
                r2[u].y = s1[u] ? 1.f : r2[u].y;
            }
            D2[u] = __fmul2_rn(r2[u], __fmul2_rn(I[u].dk, make_float2(C.z, C.w))); // D log2(e)
        }
        // a step whose pairs all have D >= 18: 1/f = 1/r, no exponential, no
        // dE/dR term (see kGbFarD2)
        const bool far = !MASKED && !SALT &&
                         __all_sync(0xffffffffu, fminf(fminf(D2[0].x, D2[0].y), fminf(D2[1].x, D2[1].y)) >= kGbFarD2);
        if (far) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float2 fi = make_float2(rsqrt_ftz(r2[u].x), rsqrt_ftz(r2[u].y));
                const float2 qq = __fmul2_rn(I[u].q, qj);
                ei[u] = __ffma2_rn(qq, fi, ei[u]);
                if (BACKWARD) {
                    ai[u][1] = __ffma2_rn(qj, fi, ai[u][1]);
                    aj[1] = __ffma2_rn(I[u].q, fi, aj[1]);
                    const float2 g2 = __fmul2_rn(tau2, __fmul2_rn(qq, __fmul2_rn(__fmul2_rn(fi, fi), fi)));
                    ai[u][2] = __ffma2_rn(g2, dx[u], ai[u][2]);
                    ai[u][3] = __ffma2_rn(g2, dy[u], ai[u][3]);
                    ai[u][4] = __ffma2_rn(g2, dz[u], ai[u][4]);
                    aj[2] = __ffma2_rn(g2, dx[u], aj[2]); // the partner's gradient is minus this sum
                    aj[3] = __ffma2_rn(g2, dy[u], aj[3]);
                    aj[4] = __ffma2_rn(g2, dz[u], aj[4]);
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float2 e = make_float2(exp2_ftz(-D2[u].x), exp2_ftz(-D2[u].y));
                const float2 fa = __ffma2_rn(__fmul2_rn(I[u].R, Rj), e, r2[u]);
                float2 fi = make_float2(rsqrt_ftz(fa.x), rsqrt_ftz(fa.y));
                if (MASKED) {
                    fi.x = s0[u] ? 0.f : fi.x;
                    fi.y = s1[u] ? 0.f : fi.y;
                }
                const float2 qq = __fmul2_rn(I[u].q, qj);
                float2 tf = one, td = one;
                if (SALT) {
                    const float2 f = __fmul2_rn(fa, fi); // effective distance
                    const float2 es = __fmul2_rn(ieo2, make_float2(exp2_ftz(-kl * f.x), exp2_ftz(-kl * f.y)));
                    tf = __ffma2_rn(es, mone, ie);                                 // tau(f)
                    td = __ffma2_rn(__fmul2_rn(kap2, f), __fmul2_rn(es, mone), tf); // taud(f)
                }
                const float2 fit = SALT ? __fmul2_rn(fi, tf) : fi; // tau(f) / f (tau factored out without salt)
                ei[u] = __ffma2_rn(qq, fit, ei[u]);
                if (BACKWARD) {
                    const float2 qf3 = __fmul2_rn(qq, __fmul2_rn(__fmul2_rn(fi, fi), fi));
                    const float2 qfe = __fmul2_rn(qf3, e);
                    float2 t = __fmul2_rn(qfe, __ffma2_rn(D2[u], ln2, one));
                    if (SALT) t = __fmul2_rn(t, td);
                    ai[u][0] = __ffma2_rn(t, Rj, ai[u][0]);
                    aj[0] = __ffma2_rn(t, I[u].R, aj[0]);
                    ai[u][1] = __ffma2_rn(qj, fit, ai[u][1]);
                    aj[1] = __ffma2_rn(I[u].q, fit, aj[1]);
                    // tau qf3 (1 - e/4); with salt taud(f) in place of tau
                    const float2 g2 = SALT ? __fmul2_rn(td, __ffma2_rn(mone, __fmul2_rn(q25, qfe), qf3))
                                           : __ffma2_rn(mtau4, qfe, __fmul2_rn(tau2, qf3));
                    ai[u][2] = __ffma2_rn(g2, dx[u], ai[u][2]);
                    ai[u][3] = __ffma2_rn(g2, dy[u], ai[u][3]);
                    ai[u][4] = __ffma2_rn(g2, dz[u], ai[u][4]);
                    aj[2] = __ffma2_rn(g2, dx[u], aj[2]); // the partner's gradient is minus this sum
                    aj[3] = __ffma2_rn(g2, dy[u], aj[3]);
                    aj[4] = __ffma2_rn(g2, dz[u], aj[4]);
                }
            }
        }
        if (BACKWARD) {
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                aj[c].x = __shfl_sync(0xffffffffu, aj[c].x, src);
                aj[c].y = __shfl_sync(0xffffffffu, aj[c].y, src);
            }
        }
    }
}

template <bool BACKWARD, bool SALT>
__global__ void __launch_bounds__(kGT, 5) k_gpair_sym(SView g) {
    __shared__ GpJs sj[kGG / 2];
    __shared__ float red[kGG][4][kGJ][5];
    __shared__ long long sfx[5][kGI]; // i-side sums, component-major (conflict-free)
    __shared__ double ered[kGT / 32];
    const GItem it = gitem(g);
    if (!it.ok) return;
    const int n = g.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* X = g.x + (size_t)it.rep * n * 3;
    const float* Q = g.q + (size_t)it.rep * n;
    const size_t base = (size_t)it.rep * n;
    const float sqk = g.sqk32, tau = g.tau32, iei = g.iei32, ieo = g.ieo32, kap = g.kap32;
    int ii[2];
    bool vi[2];
    GpI2 I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < n;
        const int i = vi[u] ? ii[u] : it.i0;
        const float R = vi[u] ? (float)g.R[base + i] : 1.f;
        I[u].x = splat<float2>(vi[u] ? X[3 * i] : -kFar);
        I[u].y = splat<float2>(vi[u] ? X[3 * i + 1] : -kFar);
        I[u].z = splat<float2>(vi[u] ? X[3 * i + 2] : -kFar);
        I[u].q = splat<float2>(vi[u] ? Q[i] * sqk : 0.f);
        I[u].R = splat<float2>(R);
        I[u].dk = splat<float2>((0.25f * kLog2e) * __frcp_rn(R));
#pragma unroll
        for (int c = 0; c < 5; ++c) sfx[c][warp * 64 + u * 32 + lane] = 0;
    }
    KSum<float> egb;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kGG) {
        const int ng = min(kGG, it.jt1 - g0), npair = (ng + 1) >> 1;
        __syncthreads();
        // stage the tile pairs: thread (pair, copy, entry) writes whole rows
        for (int q = tid; q < npair * 2 * kGJ; q += kGT) {
            const int pr = q >> 6, cpy = (q >> 5) & 1, e = q & 31;
            float v[2][6];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gt = 2 * pr + h, j = (g0 + gt) * kGJ + e;
                if (gt < ng && j < n) {
                    const float R = (float)g.R[base + j];
                    v[h][0] = -X[3 * j]; v[h][1] = -X[3 * j + 1]; v[h][2] = -X[3 * j + 2];
                    v[h][3] = Q[j] * sqk; v[h][4] = R; v[h][5] = __frcp_rn(R);
                } else { // padding: far away, no charge
                    v[h][0] = kFar; v[h][1] = kFar; v[h][2] = kFar;
                    v[h][3] = 0.f; v[h][4] = 1.f; v[h][5] = 1.f;
                }
            }
            GpJs& S = sj[pr];
            const int r = e + cpy * kGJ;
            S.a[r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
            S.b[r] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
            S.c[r] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
        }
        __syncthreads();
        // i-side partials of the staged group in FP32 (tile pairs in turn, halves
        // = even / odd tiles), one fixed-point conversion per group; groups are
        // aligned runs of kGG j-tiles, whatever the item's chunk
        float2 ai[2][5];
#pragma unroll
        for (int c = 0; c < 5; ++c) ai[0][c] = ai[1][c] = make_float2(0.f, 0.f);
        for (int pr = 0; pr < npair; ++pr) {
            float2 aj[5], ei[2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
            for (int c = 0; c < 5; ++c) aj[c] = make_float2(0.f, 0.f);
            uint32_t sk[2][2] = {{0u, 0u}, {0u, 0u}};
            bool masked = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jt = g0 + 2 * pr + h;
                if (jt < it.jt1 && gmasked(jt, it.i0, n)) {
                    masked = true;
#pragma unroll
                    for (int u = 0; u < 2; ++u) sk[u][h] = gskip(ii[u], vi[u], jt * kGJ, n);
                }
            }
            if (masked) gpair_tile<true, BACKWARD, SALT>(sj[pr], lane, I, ai, aj, ei, sk, tau, iei, ieo, kap);
            else gpair_tile<false, BACKWARD, SALT>(sj[pr], lane, I, ai, aj, ei, sk, tau, iei, ieo, kap);
            // energy: plain per-tile sums, compensated across tiles
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                egb.add(ei[u].x);
                egb.add(ei[u].y);
            }
            if (BACKWARD) {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const float sgn = c >= 2 ? -1.f : 1.f;
                    red[2 * pr][warp][lane][c] = sgn * aj[c].x;
                    red[2 * pr + 1][warp][lane][c] = sgn * aj[c].y;
                }
            }
        }
        if (BACKWARD) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int row = warp * 64 + u * 32 + lane;
#pragma unroll
                for (int c = 0; c < 5; ++c) sfx[c][row] += to_fixed(ai[u][c].x + ai[u][c].y, (float)kScaleE);
            }
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
            const int row = warp * 64 + u * 32 + lane;
            const size_t a = base + ii[u];
            atomicAdd((unsigned long long*)&g.dRfix[a], (unsigned long long)sfx[0][row]);
            atomicAdd((unsigned long long*)&g.dqfix[a], (unsigned long long)sfx[1][row]);
            atomicAdd((unsigned long long*)&g.gfix[3 * a], (unsigned long long)sfx[2][row]);
            atomicAdd((unsigned long long*)&g.gfix[3 * a + 1], (unsigned long long)sfx[3][row]);
            atomicAdd((unsigned long long*)&g.gfix[3 * a + 2], (unsigned long long)sfx[4][row]);
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
        atomicAdd((unsigned long long*)&g.eacc[it.rep], (unsigned long long)__double2ll_rn(-g.tau_pair * v * kScaleE));
    }
}

// self energy; for the backward also dE/dR, c = dE/dR dR/dpsi rt/2, dE/dq
template <bool BACKWARD>
__global__ void k_gfin_c(SView g) {
    const size_t a = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= (size_t)g.n_rep * g.n) return;
    const double q = (double)g.q[a] * g.sqrt_k, R = g.R[a];
    const double esa = sa_ace(g.sa_gamma, g.sa_probe, (double)g.rho[a], R);
    const double ts = salt_tau(R, g.inv_eps_in, g.inv_eps_out, g.kappa); // tau of the self term
    const long long e = __double2ll_rn((-0.5 * ts * q * q / R + esa) * kScaleE);
    // one atomic per warp when the warp's atoms share a replica (exact integer
    // sums, so the total is the same whichever way they are grouped)
    const unsigned mask = __activemask();
    const long long rep = (long long)(a / g.n);
    const long long rep0 = __shfl_sync(mask, rep, __ffs(mask) - 1);
    if (mask == 0xffffffffu && __all_sync(mask, rep == rep0)) {
        long long t = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) atomicAdd((unsigned long long*)&g.eacc[rep], (unsigned long long)t);
    } else {
        atomicAdd((unsigned long long*)&g.eacc[rep], (unsigned long long)e);
    }
    if (!BACKWARD) return;
    const double dEdR = 0.5 * (g.tau_pair * ((double)g.dRfix[a] / kScaleE)
                               + salt_taud(R, g.inv_eps_in, g.inv_eps_out, g.kappa) * q * q / (R * R))
                      - (g.sa_gamma != 0.0 ? 6.0 * esa / R : 0.0); // no FP64 division without the term
    const double rt = (double)g.rho[a] - g.offset;
    const double gpsi = dEdR * g.gpsi[a]; // gpsi slot held dR/dpsi
    const double dq = -g.sqrt_k * (g.tau_pair * ((double)g.dqfix[a] / kScaleE) + ts * q / R);
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
// which k_gfin_out turns into dE/drho.  In the far regime dH/dr =
// -s^3 Q(y)/r^5, dH/ds = s^2 S(y)/r^4 with y = s^2/r^2, and dH/drt = 0.
// Packed over partner tiles (A, B) like the engine's passes.
struct GcI2 {
    float2 x, y, z, c, s2, s3; // the i atom's value in both halves
    float s, rt, irt;          // closed-form operands
};

struct GcJs {
    float4 a[2 * kGJ]; // (-xA, -xB, -yA, -yB)
    float4 b[2 * kGJ]; // (-zA, -zB, cA, cB)
    float4 c[2 * kGJ]; // (s2A, s2B, s3A, s3B)
    float4 n[2 * kGJ]; // (sA, sB, rtA, rtB): closed forms
    float2 m[2 * kGJ]; // (1/rtA, 1/rtB): closed forms
};

struct GcNear {
    float t, hti, htj, asi, asj;
};

// Closed forms of one pair inside r_far or in the cutoff band, out of line
// (a warp only gets here when one of its lanes has such a pair): the gradient
// factor t, dH/drt both ways, and the c-weighted dH/ds both ways.
static __device__ __noinline__ GcNear gchain_near(float r2, float rinv, float ci, float rti, float irti, float si,
                                                  float cj, float sj, float rtj, float irtj, float rc) {
    const float r = r2 * rinv;
    GcNear o;
    o.t = (ci * hct_dr_fastlog(r, rinv, rti, sj, rc) + cj * hct_dr_fastlog(r, rinv, rtj, si, rc)) * rinv;
    o.hti = hct_drt(r, rti, irti, sj, rc);
    o.htj = hct_drt(r, rtj, irtj, si, rc);
    o.asi = cj * hct_ds(r, rinv, rtj, si, rc);
    o.asj = ci * hct_ds(r, rinv, rti, sj, rc);
    return o;
}

template <bool MASKED, bool CUT>
__device__ __forceinline__ void gchain_tile(const GcJs& sj, int lane, const GcI2 (&I)[2], float2 (&ai)[2][5],
                                            float2 (&aj)[5], const uint32_t (&sk)[2][2], const PairBand& band,
                                            float* __restrict__ hti, float2* __restrict__ htj) {
    const int src = (lane + 1) & 31;
    const float skr2 = band.skr2;
    const float2 mone = splat<float2>(-1.f);
#pragma unroll 2
    for (int k = 0; k < kGJ; ++k) {
        const float4 A = sj.a[lane + k], B = sj.b[lane + k], C = sj.c[lane + k];
        const float2 cj = make_float2(B.z, B.w), s2j = make_float2(C.x, C.y), s3j = make_float2(C.z, C.w);
        float2 dx[2], dy[2], dz[2], r2[2], t[2], asi[2], asj[2], wt[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            dx[u] = __fadd2_rn(I[u].x, make_float2(A.x, A.y));
            dy[u] = __fadd2_rn(I[u].y, make_float2(A.z, A.w));
            dz[u] = __fadd2_rn(I[u].z, make_float2(B.x, B.y));
            r2[u] = __ffma2_rn(dx[u], dx[u], __ffma2_rn(dy[u], dy[u], __fmul2_rn(dz[u], dz[u])));
            if (MASKED) {
                const int jj = (lane + k) & (kGJ - 1);
                r2[u].x = ((sk[u][0] >> jj) & 1u) ? skr2 : r2[u].x;
                r2[u].y = ((sk[u][1] >> jj) & 1u) ? skr2 : r2[u].y;
            }
            const float2 rinv2 = make_float2(rcp_ftz(r2[u].x), rcp_ftz(r2[u].y));
            const float2 rinv4 = __fmul2_rn(rinv2, rinv2);
            const float2 yj = __fmul2_rn(s2j, rinv2), yi = __fmul2_rn(I[u].s2, rinv2);
            const float2 qj = hct_series_dr(yj), qi = hct_series_dr(yi);
            // t = (c_i dH_i/dr + c_j dH_j/dr) / r = -(c_i s_j^3 Q_j + c_j s_i^3 Q_i) / r^6
            const float2 term = __ffma2_rn(__fmul2_rn(I[u].c, s3j), qj, __fmul2_rn(__fmul2_rn(cj, I[u].s3), qi));
            t[u] = __fmul2_rn(term, __fmul2_rn(__fmul2_rn(rinv4, rinv2), mone));
            // c_j dH(r; rt_j, s_i)/ds = c_j s_i^2 S_i / r^4, and i <-> j, with r^-4 the
            // weight of their fused accumulate (1 for closed forms, 0 if not counted)
            asi[u] = __fmul2_rn(__fmul2_rn(cj, I[u].s2), hct_series_ds(yi));
            asj[u] = __fmul2_rn(__fmul2_rn(I[u].c, s2j), hct_series_ds(yj));
            wt[u] = rinv4;
            if (CUT) { // beyond rc + s_max nothing descreens
                const bool o0 = r2[u].x >= band.rout2, o1 = r2[u].y >= band.rout2;
                t[u].x = o0 ? 0.f : t[u].x;
                t[u].y = o1 ? 0.f : t[u].y;
                wt[u].x = o0 ? 0.f : wt[u].x;
                wt[u].y = o1 ? 0.f : wt[u].y;
            }
        }
        // closed forms only where some lane has such a pair (rare; skipped
        // pairs never get here, and dH/drt is zero in the far regime, so only
        // this branch adds to the rt sums)
        const bool nr = band_near<CUT>(r2[0].x, band) || band_near<CUT>(r2[0].y, band) ||
                        band_near<CUT>(r2[1].x, band) || band_near<CUT>(r2[1].y, band);
        if (__any_sync(0xffffffffu, nr)) {
            const float4 Nj = sj.n[lane + k];
            const float2 Mj = sj.m[lane + k];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (band_near<CUT>(r2[u].x, band)) {
                    const GcNear o = gchain_near(r2[u].x, rsqrt_ftz(r2[u].x), I[u].c.x, I[u].rt, I[u].irt,
                                                 I[u].s, B.z, Nj.x, Nj.z, Mj.x, band.rc);
                    t[u].x = o.t;
                    hti[u * 32] += o.hti;
                    htj[(lane + k) & (kGJ - 1)].x += o.htj;
                    asi[u].x = o.asi;
                    asj[u].x = o.asj;
                    wt[u].x = 1.f;
                }
                if (band_near<CUT>(r2[u].y, band)) {
                    const GcNear o = gchain_near(r2[u].y, rsqrt_ftz(r2[u].y), I[u].c.x, I[u].rt, I[u].irt,
                                                 I[u].s, B.w, Nj.y, Nj.w, Mj.y, band.rc);
                    t[u].y = o.t;
                    hti[u * 32] += o.hti;
                    htj[(lane + k) & (kGJ - 1)].y += o.htj;
                    asi[u].y = o.asi;
                    asj[u].y = o.asj;
                    wt[u].y = 1.f;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (MASKED) {
                const int jj = (lane + k) & (kGJ - 1);
                const bool s0 = (sk[u][0] >> jj) & 1u, s1 = (sk[u][1] >> jj) & 1u;
                t[u].x = s0 ? 0.f : t[u].x;
                t[u].y = s1 ? 0.f : t[u].y;
                wt[u].x = s0 ? 0.f : wt[u].x;
                wt[u].y = s1 ? 0.f : wt[u].y;
            }
            ai[u][0] = __ffma2_rn(t[u], dx[u], ai[u][0]);
            ai[u][1] = __ffma2_rn(t[u], dy[u], ai[u][1]);
            ai[u][2] = __ffma2_rn(t[u], dz[u], ai[u][2]);
            aj[0] = __ffma2_rn(t[u], dx[u], aj[0]); // the partner's gradient is minus this sum
            aj[1] = __ffma2_rn(t[u], dy[u], aj[1]);
            aj[2] = __ffma2_rn(t[u], dz[u], aj[2]);
            ai[u][4] = __ffma2_rn(asi[u], wt[u], ai[u][4]);
            aj[4] = __ffma2_rn(asj[u], wt[u], aj[4]);
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            if (c == 3) continue; // dH/drt partials are kept in shared memory (closed forms only)
            aj[c].x = __shfl_sync(0xffffffffu, aj[c].x, src);
            aj[c].y = __shfl_sync(0xffffffffu, aj[c].y, src);
        }
    }
}

template <bool CUT>
__global__ void __launch_bounds__(kGT, 4) k_gchain_sym(SView g) {
    __shared__ GcJs sj[kGG / 2];
    __shared__ float red[kGG][4][kGJ][5];
    __shared__ long long sfx[5][kGI]; // i-side sums, component-major (conflict-free)
    // dH/drt sums, which only the rare closed-form pairs feed: i side per
    // thread and atom over a staged group, partner side per warp and tile pair
    __shared__ float hti_s[kGI];
    __shared__ float2 htj_s[kGT / 32][kGJ];
    const GItem it = gitem(g);
    if (!it.ok) return;
    const int n = g.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* X = g.x + (size_t)it.rep * n * 3;
    const float* RH = g.rho + (size_t)it.rep * n;
    const size_t base = (size_t)it.rep * n;
    const float off = g.off32;
    const PairBand band = gband(g);
    int ii[2];
    bool vi[2];
    GcI2 I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < n;
        const int i = vi[u] ? ii[u] : it.i0;
        const float rt = vi[u] ? RH[i] - off : 1.f, si = vi[u] ? g.screen[i] * rt : 0.f;
        I[u].x = splat<float2>(vi[u] ? X[3 * i] : -kFar);
        I[u].y = splat<float2>(vi[u] ? X[3 * i + 1] : -kFar);
        I[u].z = splat<float2>(vi[u] ? X[3 * i + 2] : -kFar);
        I[u].c = splat<float2>(vi[u] ? (float)g.c[base + i] : 0.f);
        I[u].s2 = splat<float2>(si * si);
        I[u].s3 = splat<float2>(si * si * si);
        I[u].s = si;
        I[u].rt = rt;
        I[u].irt = 1.f / rt;
#pragma unroll
        for (int c = 0; c < 5; ++c) sfx[c][warp * 64 + u * 32 + lane] = 0;
    }
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kGG) {
        const int ng = min(kGG, it.jt1 - g0), npair = (ng + 1) >> 1;
        __syncthreads();
        // stage the tile pairs: thread (pair, copy, entry) writes whole rows
        for (int q = tid; q < npair * 2 * kGJ; q += kGT) {
            const int pr = q >> 6, cpy = (q >> 5) & 1, e = q & 31;
            float v[2][7];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gt = 2 * pr + h, j = (g0 + gt) * kGJ + e;
                if (gt < ng && j < n) {
                    const float rt = RH[j] - off;
                    v[h][0] = -X[3 * j]; v[h][1] = -X[3 * j + 1]; v[h][2] = -X[3 * j + 2];
                    v[h][3] = (float)g.c[base + j]; v[h][4] = g.screen[j] * rt; v[h][5] = rt; v[h][6] = 1.f / rt;
                } else { // padding: far away, no weight, no sphere
                    v[h][0] = kFar; v[h][1] = kFar; v[h][2] = kFar;
                    v[h][3] = 0.f; v[h][4] = 0.f; v[h][5] = 1.f; v[h][6] = 1.f;
                }
            }
            GcJs& S = sj[pr];
            const int r = e + cpy * kGJ;
            const float s2a = v[0][4] * v[0][4], s2b = v[1][4] * v[1][4];
            S.a[r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
            S.b[r] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
            S.c[r] = make_float4(s2a, s2b, s2a * v[0][4], s2b * v[1][4]);
            S.n[r] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
            S.m[r] = make_float2(v[0][6], v[1][6]);
        }
        __syncthreads();
        // i-side partials of the staged group in FP32, one conversion per group
        float2 ai[2][5];
#pragma unroll
        for (int c = 0; c < 5; ++c) ai[0][c] = ai[1][c] = make_float2(0.f, 0.f);
        hti_s[warp * 64 + lane] = 0.f;
        hti_s[warp * 64 + 32 + lane] = 0.f;
        for (int pr = 0; pr < npair; ++pr) {
            float2 aj[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) aj[c] = make_float2(0.f, 0.f);
            htj_s[warp][lane] = make_float2(0.f, 0.f);
            __syncwarp();
            uint32_t sk[2][2] = {{0u, 0u}, {0u, 0u}};
            bool masked = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jt = g0 + 2 * pr + h;
                if (jt < it.jt1 && gmasked(jt, it.i0, n)) {
                    masked = true;
#pragma unroll
                    for (int u = 0; u < 2; ++u) sk[u][h] = gskip(ii[u], vi[u], jt * kGJ, n);
                }
            }
            if (masked) gchain_tile<true, CUT>(sj[pr], lane, I, ai, aj, sk, band, &hti_s[warp * 64 + lane], htj_s[warp]);
            else gchain_tile<false, CUT>(sj[pr], lane, I, ai, aj, sk, band, &hti_s[warp * 64 + lane], htj_s[warp]);
            __syncwarp();
            aj[3] = htj_s[warp][lane]; // lane l: partner l of both tiles
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float sgn = c < 3 ? -1.f : 1.f;
                red[2 * pr][warp][lane][c] = sgn * aj[c].x;
                red[2 * pr + 1][warp][lane][c] = sgn * aj[c].y;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int row = warp * 64 + u * 32 + lane;
            ai[u][3] = make_float2(hti_s[row], 0.f);
#pragma unroll
            for (int c = 0; c < 5; ++c) sfx[c][row] += to_fixed(ai[u][c].x + ai[u][c].y, (float)kScaleE);
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
        const int row = warp * 64 + u * 32 + lane;
        const size_t a = base + ii[u];
        atomicAdd((unsigned long long*)&g.gfix[3 * a], (unsigned long long)sfx[0][row]);
        atomicAdd((unsigned long long*)&g.gfix[3 * a + 1], (unsigned long long)sfx[1][row]);
        atomicAdd((unsigned long long*)&g.gfix[3 * a + 2], (unsigned long long)sfx[2][row]);
        atomicAdd((unsigned long long*)&g.artfix[a], (unsigned long long)sfx[3][row]);
        atomicAdd((unsigned long long*)&g.asfix[a], (unsigned long long)sfx[4][row]);
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
    const double esa = sa_ace(g.sa_gamma, g.sa_probe, rho, R); // explicit rho dependence at fixed R
    const double dr = g.dEdR[a] * R * R * (1.0 / (rt * rt) - th / (rho * rho)) + g.gpsi[a] * psi / rt +
                      g.c[a] * ((double)g.artfix[a] / kScaleE) +
                      (double)g.screen[a % g.n] * ((double)g.asfix[a] / kScaleE) +
                      (esa != 0.0 ? esa * (2.0 / (rho + g.sa_probe) + 6.0 / rho) : 0.0);
    g.dx[3 * a] = (float)(up * ((double)g.gfix[3 * a] / kScaleE));
    g.dx[3 * a + 1] = (float)(up * ((double)g.gfix[3 * a + 1] / kScaleE));
    g.dx[3 * a + 2] = (float)(up * ((double)g.gfix[3 * a + 2] / kScaleE));
    g.dqo[a] = (float)(up * g.dq[a]);
    g.drho[a] = (float)(up * dr);
}

} // namespace grad
} // namespace cph
