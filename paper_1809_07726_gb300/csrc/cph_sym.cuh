// FP32 pair passes with Newton's third law: every unordered pair is evaluated
// once and its contribution goes to both atoms.
//
// Decomposition.  A CTA of 128 threads (4 warps) owns an i-tile of 256 atoms,
// two per lane (i and i + 32 within its warp's 64), and sweeps the j-tiles
// (32 atoms each) of its work item; the items of a walker cover the upper
// triangle j > i (an i-tile meets the j-tiles from its own first atom on,
// split into chunks for load balance).  Within a j-tile the 32 partners are
// staged in shared memory and visited in rotation: at step k lane l pairs its
// two atoms with partner (l + k) mod 32, and the partner-side partial sums
// travel with the partner from lane to lane by one warp shuffle per component
// and step.  After the 32 steps each lane holds the partial sums of partner l;
// the four warps' partials are added in shared memory and sent to the
// partner's int64 fixed-point accumulator with one atomic per component.  The
// i-side partials of a chunk go the same way at its end.  Fixed-point addition
// is exact and commutative, so the result does not depend on the order in
// which CTAs finish (batched and per-replica launches agree bit for bit).
//
// j-tiles that contain the diagonal (partners j <= i must be skipped) or an
// excluded partner (no Coulomb / LJ) are listed per (system, i-tile) at set-up
// and run the masked loop; all others run the unmasked loop.
//
// Far pairs.  At set-up r_far = max(s_max / 0.35, s_max + rt_max) over every
// atom (times 1 + 1e-5), so for r >= r_far every descreening integral of the
// pair is in its disjoint-sphere series regime; one comparison of r^2 then
// selects the series for both directions.  Pairs inside r_far take closed
// forms: queued per warp in the Born pass (born_tile_q), in line behind a warp
// vote in the chain-rule pass.  In the GB pass each i-atom row of a step
// whose pairs all have D = r^2 / (4 R_i R_j) >= 18 takes the far GB form
// (kGbFarD2).
#pragma once
#include "cph_device.cuh"
#include "cph_internal.h"
#include "cph_pair_tiles.cuh"
#include "cph_kernels.cuh"

namespace cph {

constexpr int kSymThreads = 128;
constexpr int kSymI = 256;    // atoms per i-tile (two per thread)
constexpr int kSymJ = kTileJ;  // atoms per j-tile
constexpr int kSymChunk = 48; // j-tiles per work item at most (default; autotuned)
constexpr int kSymG = 8;      // j-tiles staged per barrier (four tile pairs)

struct SymItem {
    int w, i0, jt0, jt1, st, pad;
};

// Tile pairs of the staged group at g0 (npair of them) that a warp passes by:
// the first pairs whose two j-tiles hold only partners j <= i of the warp's
// 64 i atoms (an i-tile starts at a multiple of kSymI atoms), or all of them
// when the warp has no atom.  Every pair there is skipped, so their partials
// are exact zeros and the warp starts at the returned pair.
__device__ __forceinline__ int first_live_pair(int i0, int warp, int N, int g0, int npair) {
    if (i0 + warp * 64 >= N) return npair;
    const int d = i0 / kSymJ + 2 * warp - g0; // tiles below g0 + d are passed by
    return d <= 0 ? 0 : min(npair, d >> 1);
}

// Non-finite partials would saturate in the float -> int64 conversion and
// vanish into a finite-looking sum, so they are flagged before converting.
__device__ __forceinline__ void red_add(long long* p, float v, int* status) {
    if (!(fabsf(v) < 1e30f)) atomicOr(status, 4);
    atomicAdd((unsigned long long*)p, (unsigned long long)to_fixed(v, (float)kScaleE));
}

__device__ __forceinline__ void fix_add(long long* p, long long v) {
    atomicAdd((unsigned long long*)p, (unsigned long long)v);
}

__device__ __forceinline__ void red_add_h(long long* p, float v, int* status) {
    if (!(fabsf(v) < 1e20f)) atomicOr(status, 4);
    atomicAdd((unsigned long long*)p, (unsigned long long)to_fixed(v, (float)kScaleH));
}

// masks of one i atom for the j-tile at j0: bit jj of `skip` = pair not
// counted here (j <= i, or no atom), bit jj of `nb` = no Coulomb/LJ (excluded
// or skipped).
__device__ __forceinline__ void sym_masks(const View& V, int P, int i, bool vi, int j0, int N,
                                          uint32_t& skip, uint32_t& nb) {
    skip = 0xffffffffu;
    nb = 0xffffffffu;
    if (!vi) return;
    const int d = i - j0; // partners j0 + jj with jj <= d are skipped
    if (d < 0) skip = 0u;
    else if (d < 31) skip = (2u << d) - 1u;
    const int nv = N - j0;
    if (nv < 32) skip |= ~((nv <= 0) ? 0u : (0xffffffffu >> (32 - nv)));
    nb = skip;
    for (int e = V.excl_off[P + i]; e < V.excl_off[P + i + 1]; ++e) {
        const int dj = V.excl_j[e] - j0;
        if (dj >= 0 && dj < 32) nb |= 1u << dj;
    }
}

// H for a pair known to be in the far regime (both directions valid)
__device__ __forceinline__ float hct_series(float rinv, float s) {
    const float x = s * rinv, y = x * x;
    return x * y * hct_series_h(y) * rinv;
}

__device__ __forceinline__ float hct_dr_series(float rinv2, float rinv, float s) {
    const float x = s * rinv, y = x * x;
    return -x * y * hct_series_dr(y) * rinv2;
}

// ============================================== operand staging (FP32)
// The pair kernels read FP32 operands only.  Positions are taken relative to
// the walker's first atom (|x| stays within the molecule's extent, so FP32
// keeps ~4e-6 A at 40 A) and rounded once per step; the charge and Born-radius
// terms are rounded once per step after the Born radii and any MC sweep.
__global__ void k_stage_x(View V, int a0, int n) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l, o = V.w_off[V.a_walker[a]];
    if (!V.w_local[V.a_walker[a]]) return;
    V.xs[a] = make_float4((float)(V.x[3 * a] - V.x[3 * o]), (float)(V.x[3 * a + 1] - V.x[3 * o + 1]),
                          (float)(V.x[3 * a + 2] - V.x[3 * o + 2]), 0.f);
}

__global__ void k_stage_gb(View V, int a0, int n) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l;
    if (!V.w_local[V.a_walker[a]]) return;
    const float R = (float)V.R[a], iR = __frcp_rn(R);
    V.gq[a] = make_float4((float)(V.q[a] * V.sqrt_k), R, iR, (0.25f * kLog2e) * iR);
}

// ====================================================== GB + Coulomb + LJ
// Packed over partner tiles: j-tiles are taken two at a time (A, B), and at
// step k lane l pairs each of its two i atoms with partner l + k of both
// tiles; the halves of every float2 belong to tile A and tile B.  The i atom's
// values sit in both halves (set once per item), partner data is staged
// tile-interleaved (SoA, 16-byte rows, no bank conflicts), and the partner
// sums travel as float2 (one shuffle per half).  Each half sees exactly the
// arithmetic of one tile, so results do not depend on how tiles are paired.
struct GbI2 {
    float2 x, y, z;
    float2 q;   // sqrt(k) q_i
    float2 R;   // Born radius
    float2 dk;  // log2(e) / (4 R_i): D log2(e) = r^2 dk_i / R_j
    float2 sg;  // sigma_i / 2
    float2 se4; // 4 sqrt(eps_i)
};

// one staged pair of j-tiles, two copies in a row (partner l + k at l + k)
struct GbJs {
    float4 a[2 * kSymJ]; // (-xA, -xB, -yA, -yB)
    float4 b[2 * kSymJ]; // (-zA, -zB, qA, qB), q = sqrt(k) q_j
    float4 c[2 * kSymJ]; // (RA, RB, 1/RA, 1/RB)
    float4 d[2 * kSymJ]; // (sigmaA/2, sigmaB/2, sqrt(epsA), sqrt(epsB))
};

// masks of the two i atoms against the tile pair: bit jj of sk = pair not
// counted, bit jj of nb = no Coulomb / LJ; [u][0] tile A, [u][1] tile B
struct GbMask {
    uint32_t sk[2][2], nb[2][2];
};

// SALT: Debye-Hueckel screening; the GB terms then carry tau(f) (energy) and
// taud(f) (derivatives) per pair, f = 1 / fi, and the finishing kernels
// apply 1 instead of tau to the pair sums.
// Far GB pairs (kGbFarD2, cph_pair_tiles.cuh): each of a step's two i-atom
// rows (u) in which every lane's two pairs are that far (0.62 of the rows of
// an 8000-atom system, against 0.52 of whole steps) takes 1/f = 1/r, no
// exponential and no dE/dR term; GB and Coulomb then combine into
// q_i q_j / (eps_out r) (kappa = 0).

template <bool MASKED, bool ENERGY, bool SALT>
__device__ __forceinline__ void gb_tile(const GbJs& sj, int lane, const GbI2 (&I)[2], float2 (&a)[2][4],
                                        float2 (&ja)[4], const GbMask& m, float tau, float iei, float kappa,
                                        float ieo, KSum<float>& egb, KSum<float>& ec, KSum<float>& elj) {
    const int src = (lane + 1) & 31;
    const float2 ln2 = splat<float2>(kLn2), one = splat<float2>(1.f), c12 = splat<float2>(12.f),
                 cm6 = splat<float2>(-6.f), mtau = splat<float2>(-tau), qtau4 = splat<float2>(0.25f * tau),
                 ie = splat<float2>(iei), mone = splat<float2>(-1.f), q25 = splat<float2>(0.25f),
                 kap2 = splat<float2>(kappa), ieo2 = splat<float2>(ieo);
    const float kl = kappa * kLog2e;
#pragma unroll 2
    for (int k = 0; k < kSymJ; ++k) {
        const float4 A = sj.a[lane + k], B = sj.b[lane + k], C = sj.c[lane + k], D = sj.d[lane + k];
        const float2 qj = make_float2(B.z, B.w), Rj = make_float2(C.x, C.y);
        float2 dx[2], dy[2], dz[2], r2[2], D2[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            dx[u] = __fadd2_rn(I[u].x, make_float2(A.x, A.y));
            dy[u] = __fadd2_rn(I[u].y, make_float2(A.z, A.w));
            dz[u] = __fadd2_rn(I[u].z, make_float2(B.x, B.y));
            r2[u] = __ffma2_rn(dx[u], dx[u], __ffma2_rn(dy[u], dy[u], __fmul2_rn(dz[u], dz[u])));
            if (MASKED) {
                const int jj = (lane + k) & (kSymJ - 1);
                r2[u].x = ((m.sk[u][0] >> jj) & 1u) ? 1.f : r2[u].x;
                r2[u].y = ((m.sk[u][1] >> jj) & 1u) ? 1.f : r2[u].y;
            }
            D2[u] = __fmul2_rn(r2[u], __fmul2_rn(I[u].dk, make_float2(C.z, C.w))); // D log2(e)
        }
        const bool vf = !MASKED && !SALT; // the far form is only taken on unmasked, salt-free tiles
        const bool f0 = vf && __all_sync(0xffffffffu, fminf(D2[0].x, D2[0].y) >= kGbFarD2);
        const bool f1 = vf && __all_sync(0xffffffffu, fminf(D2[1].x, D2[1].y) >= kGbFarD2);
        auto far_u = [&](const int u) {
                const float2 qq = __fmul2_rn(I[u].q, qj);
                const float2 ep4 = __fmul2_rn(I[u].se4, make_float2(D.z, D.w));
                const float2 rinv = make_float2(rsqrt_ftz(r2[u].x), rsqrt_ftz(r2[u].y));
                const float2 rinv2 = __fmul2_rn(rinv, rinv);
                const float2 sig = __fadd2_rn(I[u].sg, make_float2(D.x, D.y));
                const float2 sr2 = __fmul2_rn(__fmul2_rn(sig, sig), rinv2);
                const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
                const float2 l6 = __fmul2_rn(ep4, sr6);
                const float2 lj = __fmul2_rn(l6, __ffma2_rn(c12, sr6, cm6));
                // (Coulomb - tau GB) q_i q_j / r^3 = q_i q_j / (eps_out r^3)
                const float2 fs = __fmul2_rn(__ffma2_rn(__fmul2_rn(qq, rinv), ieo2, lj), rinv2);
                a[u][0] = __ffma2_rn(fs, dx[u], a[u][0]);
                a[u][1] = __ffma2_rn(fs, dy[u], a[u][1]);
                a[u][2] = __ffma2_rn(fs, dz[u], a[u][2]);
                ja[0] = __ffma2_rn(fs, dx[u], ja[0]); // the partner's force is minus this sum
                ja[1] = __ffma2_rn(fs, dy[u], ja[1]);
                ja[2] = __ffma2_rn(fs, dz[u], ja[2]);
                if (ENERGY) {
                    const float2 eg = __fmul2_rn(qq, rinv);
                    const float2 eco = __fmul2_rn(__fmul2_rn(qq, ie), rinv);
                    const float2 el = __fmul2_rn(l6, __fadd2_rn(sr6, splat<float2>(-1.f)));
                    egb.add(eg.x);
                    egb.add(eg.y);
                    ec.add(eco.x);
                    ec.add(eco.y);
                    elj.add(el.x);
                    elj.add(el.y);
                }
        };
        auto full_u = [&](const int u) {
                float2 qq = __fmul2_rn(I[u].q, qj);
                float2 ep4 = __fmul2_rn(I[u].se4, make_float2(D.z, D.w));
                if (MASKED) {
                    const int jj = (lane + k) & (kSymJ - 1);
                    const bool s0 = (m.sk[u][0] >> jj) & 1u, s1 = (m.sk[u][1] >> jj) & 1u;
                    const bool b0 = (m.nb[u][0] >> jj) & 1u, b1 = (m.nb[u][1] >> jj) & 1u;
                    qq.x = s0 ? 0.f : qq.x;
                    qq.y = s1 ? 0.f : qq.y;
                    ep4.x = b0 ? 0.f : ep4.x;
                    ep4.y = b1 ? 0.f : ep4.y;
                }
                float2 cq = __fmul2_rn(qq, ie); // sqrt(k) q_i sqrt(k) q_j / eps_in
                if (MASKED) {
                    const int jj = (lane + k) & (kSymJ - 1);
                    cq.x = ((m.nb[u][0] >> jj) & 1u) ? 0.f : cq.x;
                    cq.y = ((m.nb[u][1] >> jj) & 1u) ? 0.f : cq.y;
                }
                const float2 rinv = make_float2(rsqrt_ftz(r2[u].x), rsqrt_ftz(r2[u].y));
                const float2 rinv2 = __fmul2_rn(rinv, rinv);
                const float2 e = make_float2(exp2_ftz(-D2[u].x), exp2_ftz(-D2[u].y));
                const float2 fa = __ffma2_rn(__fmul2_rn(I[u].R, Rj), e, r2[u]);
                const float2 fi = make_float2(rsqrt_ftz(fa.x), rsqrt_ftz(fa.y));
                const float2 qf3 = __fmul2_rn(qq, __fmul2_rn(__fmul2_rn(fi, fi), fi));
                const float2 qfe = __fmul2_rn(qf3, e);
                float2 tf = one, td = one;
                if (SALT) {
                    const float2 f = __fmul2_rn(fa, fi); // effective distance
                    const float2 es = __fmul2_rn(ieo2, make_float2(exp2_ftz(-kl * f.x), exp2_ftz(-kl * f.y)));
                    tf = __ffma2_rn(es, mone, ie);                                 // tau(f)
                    td = __ffma2_rn(__fmul2_rn(kap2, f), __fmul2_rn(es, mone), tf); // taud(f)
                }
                float2 t = __fmul2_rn(qfe, __ffma2_rn(D2[u], ln2, one));
                if (SALT) t = __fmul2_rn(t, td);
                a[u][3] = __ffma2_rn(t, Rj, a[u][3]);
                ja[3] = __ffma2_rn(t, I[u].R, ja[3]);
                const float2 sig = __fadd2_rn(I[u].sg, make_float2(D.x, D.y));
                const float2 sr2 = __fmul2_rn(__fmul2_rn(sig, sig), rinv2);
                const float2 sr6 = __fmul2_rn(__fmul2_rn(sr2, sr2), sr2);
                const float2 l6 = __fmul2_rn(ep4, sr6);
                const float2 lj = __fmul2_rn(l6, __ffma2_rn(c12, sr6, cm6));
                // -tau qf3 (1 - e/4); with salt taud(f) in place of tau
                const float2 w = SALT ? __fmul2_rn(td, __ffma2_rn(q25, qfe, __fmul2_rn(mone, qf3)))
                                      : __ffma2_rn(qtau4, qfe, __fmul2_rn(mtau, qf3));
                const float2 fs = __ffma2_rn(__ffma2_rn(cq, rinv, lj), rinv2, w);
                a[u][0] = __ffma2_rn(fs, dx[u], a[u][0]);
                a[u][1] = __ffma2_rn(fs, dy[u], a[u][1]);
                a[u][2] = __ffma2_rn(fs, dz[u], a[u][2]);
                ja[0] = __ffma2_rn(fs, dx[u], ja[0]); // the partner's force is minus this sum
                ja[1] = __ffma2_rn(fs, dy[u], ja[1]);
                ja[2] = __ffma2_rn(fs, dz[u], ja[2]);
                if (ENERGY) {
                    const float2 eg = SALT ? __fmul2_rn(tf, __fmul2_rn(qq, fi)) : __fmul2_rn(qq, fi);
                    const float2 eco = __fmul2_rn(cq, rinv);
                    const float2 el = __fmul2_rn(l6, __fadd2_rn(sr6, splat<float2>(-1.f)));
                    egb.add(eg.x);
                    egb.add(eg.y);
                    ec.add(eco.x);
                    ec.add(eco.y);
                    elj.add(el.x);
                    elj.add(el.y);
                }
        };
        // one vote per i atom row (u): the four combinations keep both rows'
        // arithmetic interleaved in one branch
        if (f0 && f1) {
            far_u(0);
            far_u(1);
        } else if (f0) {
            far_u(0);
            full_u(1);
        } else if (f1) {
            full_u(0);
            far_u(1);
        } else {
            full_u(0);
            full_u(1);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ja[c].x = __shfl_sync(0xffffffffu, ja[c].x, src);
            ja[c].y = __shfl_sync(0xffffffffu, ja[c].y, src);
        }
    }
}

template <bool ENERGY, bool SALT>
__global__ void __launch_bounds__(kSymThreads, 5) k_gb_sym(const SymItem* __restrict__ items, View V) {
    __shared__ GbJs sj[kSymG / 2];
    __shared__ __align__(16) float red[kSymG][4][kSymJ][4];
    __shared__ long long sfx[4][kSymI]; // i-side fixed-point sums, component-major (conflict-free)
    __shared__ double ered[kSymThreads / 32][3];
    const SymItem it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float tau = V.tau32, iei = V.iei32, kappa = V.kappa32, ieo = V.ieo32;
    int ii[2];
    bool vi[2];
    GbI2 I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < N;
        const int i = vi[u] ? ii[u] : it.i0;
        const float4 xi = V.xs[A + i], gi = V.gq[A + i];
        const float2 li = V.plj32[P + i];
        I[u].x = splat<float2>(vi[u] ? xi.x : -kFarF);
        I[u].y = splat<float2>(vi[u] ? xi.y : -kFarF);
        I[u].z = splat<float2>(vi[u] ? xi.z : -kFarF);
        I[u].q = splat<float2>(vi[u] ? gi.x : 0.f);
        I[u].R = splat<float2>(vi[u] ? gi.y : 1.f);
        I[u].dk = splat<float2>(vi[u] ? gi.w : 1.f);
        I[u].sg = splat<float2>(vi[u] ? li.x : 0.f);
        I[u].se4 = splat<float2>(vi[u] ? 4.f * li.y : 0.f);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) sfx[c][warp * 64 + u * 32 + lane] = 0;
    KSum<float> egb, ec, elj;
    int mp = V.smt_off[it.st];
    const int me = V.smt_off[it.st + 1];
    while (mp < me && V.smt_list[mp] < it.jt0) ++mp;
    int next = mp < me ? V.smt_list[mp] : 0x7fffffff;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kSymG) {
        const int ng = min(kSymG, it.jt1 - g0), npair = (ng + 1) >> 1;
        __syncthreads();
        // stage the tile pairs: thread (pair, copy, entry) writes whole rows
        for (int q = tid; q < npair * 2 * kSymJ; q += kSymThreads) {
            const int pr = q >> 6, cpy = (q >> 5) & 1, e = q & 31;
            {
                float v[2][8];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int g = 2 * pr + h, j = (g0 + g) * kSymJ + e;
                    if (g < ng && j < N) {
                        const float4 xj = V.xs[A + j], gj = V.gq[A + j];
                        const float2 lj = V.plj32[P + j];
                        v[h][0] = -xj.x; v[h][1] = -xj.y; v[h][2] = -xj.z; v[h][3] = gj.x;
                        v[h][4] = gj.y; v[h][5] = gj.z; v[h][6] = lj.x; v[h][7] = lj.y;
                    } else { // padding: far away, no charge, no LJ
                        v[h][0] = -kFarF; v[h][1] = -kFarF; v[h][2] = -kFarF; v[h][3] = 0.f;
                        v[h][4] = 1.f; v[h][5] = 1.f; v[h][6] = 0.f; v[h][7] = 0.f;
                    }
                }
                GbJs& S = sj[pr];
                const int r = e + cpy * kSymJ;
                S.a[r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
                S.b[r] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
                S.c[r] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
                S.d[r] = make_float4(v[0][6], v[1][6], v[0][7], v[1][7]);
            }
        }
        __syncthreads();
        // i-side partials of the whole staged group, summed in FP32 in a fixed
        // order (tile pairs in turn, halves = even / odd tiles) and converted to
        // fixed point once per group: groups are the aligned runs of kSymG
        // j-tiles (items start at a multiple of kSymG tiles and span a multiple
        // of it), so the sums do not depend on the item's chunking
        float2 acc[2][4] = {{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}},
                            {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}};
        for (int pr = 0; pr < npair; ++pr) {
            const int jtA = g0 + 2 * pr; // tile B (jtA + 1) may lie past the item: padding
            float2 ja[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            GbMask m = {};
            bool masked = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jt = jtA + h;
                if (jt < it.jt1 && jt == next) {
                    ++mp;
                    next = mp < me ? V.smt_list[mp] : 0x7fffffff;
                    masked = true;
#pragma unroll
                    for (int u = 0; u < 2; ++u) sym_masks(V, P, ii[u], vi[u], jt * kSymJ, N, m.sk[u][h], m.nb[u][h]);
                }
            }
            if (masked) gb_tile<true, ENERGY, SALT>(sj[pr], lane, I, acc, ja, m, tau, iei, kappa, ieo, egb, ec, elj);
            else gb_tile<false, ENERGY, SALT>(sj[pr], lane, I, acc, ja, m, tau, iei, kappa, ieo, egb, ec, elj);
            // lane l now holds the partials of partner l of both tiles
            *reinterpret_cast<float4*>(red[2 * pr][warp][lane]) = make_float4(-ja[0].x, -ja[1].x, -ja[2].x, ja[3].x);
            *reinterpret_cast<float4*>(red[2 * pr + 1][warp][lane]) = make_float4(-ja[0].y, -ja[1].y, -ja[2].y, ja[3].y);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                sfx[c][warp * 64 + u * 32 + lane] += to_fixed(acc[u][c].x + acc[u][c].y, (float)kScaleE);
        __syncthreads();
        // add the four warps' partials of every staged partner and send them
        for (int v = tid; v < ng * kSymJ * 4; v += kSymThreads) {
            const int g = v / (kSymJ * 4), j = (v >> 2) & (kSymJ - 1), c = v & 3;
            const float sum = red[g][0][j][c] + red[g][1][j][c] + red[g][2][j][c] + red[g][3][j][c];
            const int jg = (g0 + g) * kSymJ + j;
            if (jg < N) {
                long long* dst = (c < 3) ? &V.Ffix[3 * (A + jg) + c] : &V.dRfix[A + jg];
                red_add(dst, sum, V.status);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (vi[u]) {
            const int r = warp * 64 + u * 32 + lane;
            fix_add(&V.Ffix[3 * (A + ii[u])], sfx[0][r]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 1], sfx[1][r]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 2], sfx[2][r]);
            fix_add(&V.dRfix[A + ii[u]], sfx[3][r]);
        }
    }
    if (ENERGY) {
        // compensated lane sums, reduced in FP64
        double e0 = (double)egb.s - (double)egb.c, e1 = (double)ec.s - (double)ec.c,
               e2 = (double)elj.s - (double)elj.c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e0 += __shfl_down_sync(0xffffffffu, e0, o);
            e1 += __shfl_down_sync(0xffffffffu, e1, o);
            e2 += __shfl_down_sync(0xffffffffu, e2, o);
        }
        if (lane == 0) {
            ered[warp][0] = e0;
            ered[warp][1] = e1;
            ered[warp][2] = e2;
        }
        __syncthreads();
        if (tid < 3) {
            double v = 0.0;
            for (int q = 0; q < kSymThreads / 32; ++q) v += ered[q][tid];
            // GB pairs carry -tau (with salt, tau(f) per pair and -1 here); Coulomb already has
            // 1/eps_in, LJ its factor 4
            const double scale = (tid == 0) ? -V.tau_pair : 1.0;
            atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + tid],
                      (unsigned long long)__double2ll_rn(scale * v * kScaleE));
        }
    }
}

// dE/dR (fixed point) -> chain weights c_i; GB self energy
template <bool ENERGY>
__global__ void k_fin_c(View V, int a0, int n) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l;
    const int w = V.a_walker[a];
    if (V.sys_ordered[V.w_sys[w]] || !V.w_local[w]) return; // ordered passes finish their atoms themselves
    const int P = V.sys_poff[V.w_sys[w]] + (a - V.w_off[w]);
    const double q = V.q[a] * V.sqrt_k, R = V.R[a];
    const double esa = sa_ace(V.sa_gamma, V.sa_probe, V.rho[P], R);
    const double dEdR = 0.5 * (V.tau_pair * ((double)V.dRfix[a] / kScaleE)
                               + salt_taud(R, V.inv_eps_in, V.inv_eps_out, V.kappa) * q * q / (R * R))
                      - (V.sa_gamma != 0.0 ? 6.0 * esa / R : 0.0); // no FP64 division without the term
    const double c = dEdR * V.dRdpsi[a] * 0.5 * V.rt[P];
    V.c[a] = c;
    V.c32[a] = (float)c;
    if (ENERGY)
        atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 0],
                  (unsigned long long)__double2ll_rn((-0.5 * salt_tau(R, V.inv_eps_in, V.inv_eps_out, V.kappa)
                                                      * q * q / R + esa) * kScaleE));
}

// ========================================================= chain rule
// F_i -= sum_k c_k dI_k/dx_i with c = dE/dR dR/dpsi rt/2: for a pair, the force
// along the separation is t = -(c_i dH(r, rt_i, s_j)/dr + c_j dH(r, rt_j, s_i)/dr) / r.
// In the far regime dH/dr = -s^3 Q(s^2/r^2) / r^5, so
// t = (c_i s_j^3 Q(s_j^2/r^2) + c_j s_i^3 Q(s_i^2/r^2)) / r^6.
// Packed over partner tiles like the GB pass.
struct ChI2 {
    float2 x, y, z, c, s2, s3; // the i atom's value in both halves
    float s, rt;               // closed-form operands
};

struct ChJs {
    float4 a[2 * kSymJ]; // (-xA, -xB, -yA, -yB)
    float4 b[2 * kSymJ]; // (-zA, -zB, cA, cB)
    float4 c[2 * kSymJ]; // (s2A, s2B, s3A, s3B)
    float4 n[2 * kSymJ]; // (sA, sB, rtA, rtB): closed forms
};

// Closed-form force weight t of one pair inside r_far (or in the cutoff
// band).  Inlined: unlike born_near, this is measured faster in line (the
// chain tile keeps fewer values live across the branch).
__device__ __forceinline__ float chain_near(float r2, float rinv, float c_i, float rt_i, float s_i, float c_j,
                                         float s_j, float rt_j, float rc) {
    const float r = r2 * rinv;
    const float g = c_i * hct_dr_fastlog(r, rinv, rt_i, s_j, rc) + c_j * hct_dr_fastlog(r, rinv, rt_j, s_i, rc);
    return -g * rinv;
}

template <bool MASKED, bool CUT>
__device__ __forceinline__ void chain_tile(const ChJs& sj, int lane, const ChI2 (&I)[2], float2 (&a)[2][3],
                                           float2 (&ja)[3], const uint32_t (&sk)[2][2], const PairBand& band) {
    const int src = (lane + 1) & 31;
    const float skr2 = band.skr2;
#pragma unroll 2
    for (int k = 0; k < kSymJ; ++k) {
        const float4 A = sj.a[lane + k], B = sj.b[lane + k], C = sj.c[lane + k];
        const float2 cj = make_float2(B.z, B.w), s2j = make_float2(C.x, C.y), s3j = make_float2(C.z, C.w);
        float2 dx[2], dy[2], dz[2], r2[2], t[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            dx[u] = __fadd2_rn(I[u].x, make_float2(A.x, A.y));
            dy[u] = __fadd2_rn(I[u].y, make_float2(A.z, A.w));
            dz[u] = __fadd2_rn(I[u].z, make_float2(B.x, B.y));
            r2[u] = __ffma2_rn(dx[u], dx[u], __ffma2_rn(dy[u], dy[u], __fmul2_rn(dz[u], dz[u])));
            if (MASKED) { // skipped pairs stay off the closed-form branch
                const int jj = (lane + k) & (kSymJ - 1);
                r2[u].x = ((sk[u][0] >> jj) & 1u) ? skr2 : r2[u].x;
                r2[u].y = ((sk[u][1] >> jj) & 1u) ? skr2 : r2[u].y;
            }
            const float2 rinv2 = make_float2(rcp_ftz(r2[u].x), rcp_ftz(r2[u].y));
            const float2 qj = hct_series_dr(__fmul2_rn(s2j, rinv2));
            const float2 qi = hct_series_dr(__fmul2_rn(I[u].s2, rinv2));
            const float2 term = __ffma2_rn(__fmul2_rn(I[u].c, s3j), qj, __fmul2_rn(__fmul2_rn(cj, I[u].s3), qi));
            const float2 rinv4 = __fmul2_rn(rinv2, rinv2);
            t[u] = __fmul2_rn(term, __fmul2_rn(rinv4, rinv2));
            if (CUT) { // beyond rc + s_max nothing descreens
                t[u].x = r2[u].x >= band.rout2 ? 0.f : t[u].x;
                t[u].y = r2[u].y >= band.rout2 ? 0.f : t[u].y;
            }
        }
        // closed forms only where some lane has such a pair (rare)
        const bool nr = band_near<CUT>(r2[0].x, band) || band_near<CUT>(r2[0].y, band) ||
                        band_near<CUT>(r2[1].x, band) || band_near<CUT>(r2[1].y, band);
        if (__any_sync(0xffffffffu, nr)) {
            const float4 Nj = sj.n[lane + k];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (band_near<CUT>(r2[u].x, band))
                    t[u].x = chain_near(r2[u].x, rsqrt_ftz(r2[u].x), I[u].c.x, I[u].rt, I[u].s, B.z, Nj.x, Nj.z,
                                        band.rc);
                if (band_near<CUT>(r2[u].y, band))
                    t[u].y = chain_near(r2[u].y, rsqrt_ftz(r2[u].y), I[u].c.x, I[u].rt, I[u].s, B.w, Nj.y, Nj.w,
                                        band.rc);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (MASKED) {
                const int jj = (lane + k) & (kSymJ - 1);
                t[u].x = ((sk[u][0] >> jj) & 1u) ? 0.f : t[u].x;
                t[u].y = ((sk[u][1] >> jj) & 1u) ? 0.f : t[u].y;
            }
            a[u][0] = __ffma2_rn(t[u], dx[u], a[u][0]);
            a[u][1] = __ffma2_rn(t[u], dy[u], a[u][1]);
            a[u][2] = __ffma2_rn(t[u], dz[u], a[u][2]);
            ja[0] = __ffma2_rn(t[u], dx[u], ja[0]); // the partner's force is minus this sum
            ja[1] = __ffma2_rn(t[u], dy[u], ja[1]);
            ja[2] = __ffma2_rn(t[u], dz[u], ja[2]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ja[c].x = __shfl_sync(0xffffffffu, ja[c].x, src);
            ja[c].y = __shfl_sync(0xffffffffu, ja[c].y, src);
        }
    }
}

template <bool CUT>
__global__ void __launch_bounds__(kSymThreads, 5) k_chain_sym(const SymItem* __restrict__ items, View V) {
    __shared__ ChJs sj[kSymG / 2];
    __shared__ __align__(16) float red[kSymG][4][kSymJ][4]; // component 3 unused (vector stores)
    __shared__ long long sfx[3][kSymI]; // i-side fixed-point sums, component-major (conflict-free)
    const SymItem it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PairBand band = pair_band(V.rfar2, V.smax32, (float)V.rgbmax);
    int ii[2];
    bool vi[2];
    ChI2 I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < N;
        const int i = vi[u] ? ii[u] : it.i0;
        const float4 xi = V.xs[A + i], pi = V.pb32[P + i];
        const float si = vi[u] ? pi.x : 0.f;
        I[u].x = splat<float2>(vi[u] ? xi.x : -kFarF);
        I[u].y = splat<float2>(vi[u] ? xi.y : -kFarF);
        I[u].z = splat<float2>(vi[u] ? xi.z : -kFarF);
        I[u].c = splat<float2>(vi[u] ? V.c32[A + i] : 0.f);
        I[u].s2 = splat<float2>(si * si);
        I[u].s3 = splat<float2>(si * si * si);
        I[u].s = si;
        I[u].rt = vi[u] ? pi.y : 1.f;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) sfx[c][warp * 64 + u * 32 + lane] = 0;
    int mp = V.smt_off[it.st];
    const int me = V.smt_off[it.st + 1];
    while (mp < me && V.smt_list[mp] < it.jt0) ++mp;
    int next = mp < me ? V.smt_list[mp] : 0x7fffffff;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kSymG) {
        const int ng = min(kSymG, it.jt1 - g0), npair = (ng + 1) >> 1;
        __syncthreads();
        // stage the tile pairs: thread (pair, copy, entry) writes whole rows
        for (int q = tid; q < npair * 2 * kSymJ; q += kSymThreads) {
            const int pr = q >> 6, cpy = (q >> 5) & 1, e = q & 31;
            {
                float v[2][6];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int g = 2 * pr + h, j = (g0 + g) * kSymJ + e;
                    if (g < ng && j < N) {
                        const float4 xj = V.xs[A + j], pj = V.pb32[P + j];
                        v[h][0] = -xj.x; v[h][1] = -xj.y; v[h][2] = -xj.z; v[h][3] = V.c32[A + j];
                        v[h][4] = pj.x; v[h][5] = pj.y;
                    } else { // padding: far away, no weight, no sphere
                        v[h][0] = -kFarF; v[h][1] = -kFarF; v[h][2] = -kFarF; v[h][3] = 0.f;
                        v[h][4] = 0.f; v[h][5] = 1.f;
                    }
                }
                ChJs& S = sj[pr];
                const int r = e + cpy * kSymJ;
                const float s2a = v[0][4] * v[0][4], s2b = v[1][4] * v[1][4];
                S.a[r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
                S.b[r] = make_float4(v[0][2], v[1][2], v[0][3], v[1][3]);
                S.c[r] = make_float4(s2a, s2b, s2a * v[0][4], s2b * v[1][4]);
                S.n[r] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
            }
        }
        __syncthreads();
        // i-side partials of the staged group in FP32, one conversion per group
        // (aligned runs of kSymG j-tiles: independent of the item's chunking)
        float2 acc[2][3] = {{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}};
        for (int pr = 0; pr < npair; ++pr) {
            const int jtA = g0 + 2 * pr;
            float2 ja[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            uint32_t sk[2][2] = {{0u, 0u}, {0u, 0u}};
            bool masked = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jt = jtA + h;
                if (jt < it.jt1 && jt == next) {
                    ++mp;
                    next = mp < me ? V.smt_list[mp] : 0x7fffffff;
                    masked = true;
                    uint32_t nbm;
#pragma unroll
                    for (int u = 0; u < 2; ++u) sym_masks(V, P, ii[u], vi[u], jt * kSymJ, N, sk[u][h], nbm);
                }
            }
            if (masked) chain_tile<true, CUT>(sj[pr], lane, I, acc, ja, sk, band);
            else chain_tile<false, CUT>(sj[pr], lane, I, acc, ja, sk, band);
            *reinterpret_cast<float4*>(red[2 * pr][warp][lane]) = make_float4(-ja[0].x, -ja[1].x, -ja[2].x, 0.f);
            *reinterpret_cast<float4*>(red[2 * pr + 1][warp][lane]) = make_float4(-ja[0].y, -ja[1].y, -ja[2].y, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                sfx[c][warp * 64 + u * 32 + lane] += to_fixed(acc[u][c].x + acc[u][c].y, (float)kScaleE);
        __syncthreads();
        for (int v = tid; v < ng * kSymJ * 3; v += kSymThreads) {
            const int g = v / (kSymJ * 3), rem = v % (kSymJ * 3), j = rem / 3, c = rem % 3;
            const float sum = red[g][0][j][c] + red[g][1][j][c] + red[g][2][j][c] + red[g][3][j][c];
            const int jg = (g0 + g) * kSymJ + j;
            if (jg < N) red_add(&V.Ffix[3 * (A + jg) + c], sum, V.status);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (vi[u]) {
            const int r = warp * 64 + u * 32 + lane;
            fix_add(&V.Ffix[3 * (A + ii[u])], sfx[0][r]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 1], sfx[1][r]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 2], sfx[2][r]);
        }
    }
}

// Bonded terms, one thread per (walker, term), FP64: each bond or angle is
// evaluated once and its forces on its two or three atoms are stored in the
// per-term buffer (the atoms gather them in a fixed order in k_final_forces,
// so the sum stays deterministic); energies per walker in fixed point.
constexpr int kBondedThreads = 256;

template <bool ENERGY>
__global__ void __launch_bounds__(kBondedThreads) k_bonded_terms(View V, int w0) {
    __shared__ double re[kBondedThreads / 32][2];
    const int w = w0 + blockIdx.y;
    const int s = V.w_sys[w], A = V.w_off[w];
    if (V.sys_ordered[s] || !V.w_local[w]) return; // bonded terms of the ordered passes are in k_chain
    const int b0 = V.sys_bond_off[s], nb = V.sys_bond_off[s + 1] - b0;
    const int a0 = V.sys_ang_off[s], na = V.sys_ang_off[s + 1] - a0;
    const int t = blockIdx.x * kBondedThreads + threadIdx.x;
    float* buf = V.tforce + V.w_tf_off[w];
    const double* x = V.x;
    double eb = 0.0, ea = 0.0;
    // the FP32-mode term arithmetic of bond_term32 / angle_term32
    if (t < nb) {
        const int b = b0 + t;
        const int i = V.bond_ij[2 * b], j = V.bond_ij[2 * b + 1];
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = x[3 * (A + i) + c] - x[3 * (A + j) + c];
        float g, e;
        bond_term32(d, V.bond_r0[b], V.bond_k[b], g, e);
        for (int c = 0; c < 3; ++c) {
            const float f = g * (float)d[c];
            buf[6 * t + c] = -f;
            buf[6 * t + 3 + c] = f;
        }
        eb = (double)e;
    } else if (t < nb + na) {
        const int la = t - nb, a = a0 + la;
        const int ia = V.ang_ijk[3 * a], ib = V.ang_ijk[3 * a + 1], ic = V.ang_ijk[3 * a + 2];
        double u[3], v[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = x[3 * (A + ia) + c] - x[3 * (A + ib) + c];
            v[c] = x[3 * (A + ic) + c] - x[3 * (A + ib) + c];
        }
        float gi[3], gk[3], e;
        angle_term32(u, v, V.ang_cs0[a], V.ang_k[a], gi, gk, e);
        float* o = buf + 6 * (size_t)nb + 9 * (size_t)la;
        for (int c = 0; c < 3; ++c) {
            o[c] = -gi[c];
            o[3 + c] = gi[c] + gk[c];
            o[6 + c] = -gk[c];
        }
        ea = (double)e;
    }
    if (ENERGY) {
#pragma unroll
        for (int of = 16; of > 0; of >>= 1) {
            eb += __shfl_down_sync(0xffffffffu, eb, of);
            ea += __shfl_down_sync(0xffffffffu, ea, of);
        }
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        if (lane == 0) {
            re[wp][0] = eb;
            re[wp][1] = ea;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            double v = 0.0;
            for (int q = 0; q < kBondedThreads / 32; ++q) v += re[q][threadIdx.x];
            if (v != 0.0)
                atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 3 + threadIdx.x],
                          (unsigned long long)__double2ll_rn(v * kScaleE));
        }
    }
}

// total force: fixed-point pair forces + the atom's bonded-term forces
__global__ void k_final_forces(View V, int a0, int n) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l;
    const int w = V.a_walker[a];
    const int s = V.w_sys[w];
    if (V.sys_ordered[s] || !V.w_local[w]) return;
    const int A = V.w_off[w], li = a - A, P = V.sys_poff[s];
    // the atom's bonded-term forces (FP32, a few terms) are summed in FP32 and
    // added once per component: FP64 conversions and additions are scarce
    float fb[3] = {0.f, 0.f, 0.f};
    const float* buf = V.tforce + V.w_tf_off[w];
    const int b0 = V.sys_bond_off[s], nb = V.sys_bond_off[s + 1] - b0, an0 = V.sys_ang_off[s];
    for (int e = V.bond_off[P + li]; e < V.bond_off[P + li + 1]; ++e) {
        const int b = V.bond_idx[e];
        const int role = (V.bond_ij[2 * b] == li) ? 0 : 1;
        const float* o = buf + 6 * (b - b0) + 3 * role;
        for (int c = 0; c < 3; ++c) fb[c] += o[c];
    }
    for (int e = V.ang_off[P + li]; e < V.ang_off[P + li + 1]; ++e) {
        const int ag = V.ang_idx[e];
        const int role = (V.ang_ijk[3 * ag] == li) ? 0 : ((V.ang_ijk[3 * ag + 1] == li) ? 1 : 2);
        const float* o = buf + 6 * (size_t)nb + 9 * (size_t)(ag - an0) + 3 * role;
        for (int c = 0; c < 3; ++c) fb[c] += o[c];
    }
    double F[3];
    for (int c = 0; c < 3; ++c) {
        F[c] = (double)V.Ffix[3 * a + c] / kScaleE + (double)fb[c];
        V.F[3 * a + c] = F[c];
    }
    if (!(isfinite(F[0]) && isfinite(F[1]) && isfinite(F[2]))) atomicOr(V.status, 1);
}

// ========================================================= Born radii
// Tile arithmetic (BoI2, BoJs, born_tile) in cph_pair_tiles.cuh.  The engine's
// pass keeps the closed forms out of the tile loop: a pair inside r_far (or
// in the cutoff band) gets weight 0 there and is queued, per warp, as
// (tile pair, half, partner, i slot); the warp evaluates its queue 32 pairs
// at a time with every lane busy (once 64 are pending, and at the end of each
// staged group), adding both integrals of each queued pair in int64 fixed
// point to shared sums (order independent).  A flush recomputes r^2 with the
// tile's own arithmetic, so the near/far decision is the same.
constexpr int kNearQ = 192; // queue entries per warp: flushed at >= 64; a step adds <= 128

struct BoNear {
    uint32_t q[kSymThreads / 32][kNearQ]; // lane | u << 5 | partner << 6 | half << 11 | pair << 12
    float4 ix[kSymThreads / 32][64];      // the warp's i atoms (x, y, z, s), slot u * 32 + lane
    float2 it[kSymThreads / 32][64];      // (rt, 1/rt)
    long long ihx[kSymThreads / 32][64];  // i-side sums of queued pairs (2^40 fixed point)
    long long jhx[kSymG][kSymJ];          // partner-side sums of the staged group
};

__device__ __noinline__ void born_flush(const BoJs* sj, BoNear& nb, int warp, int lane, int n, PairBand band,
                                        int* status) {
    for (int e = lane; e < n; e += 32) {
        const uint32_t q = nb.q[warp][e];
        const int l = q & 31u, u = (q >> 5) & 1u, jj = (q >> 6) & 31u, h = (q >> 11) & 1u, pr = q >> 12;
        const int slot = u * 32 + l;
        const float4 xi = nb.ix[warp][slot];
        const float2 ti = nb.it[warp][slot];
        const BoJs& S = sj[pr];
        const float4 A = S.a[jj], B = S.b[jj], C = S.c[jj], Nj = S.n[jj];
        const float dx = xi.x + (h ? A.y : A.x), dy = xi.y + (h ? A.w : A.z), dz = xi.z + (h ? B.y : B.x);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float2 hv = born_near(r2, rsqrt_ftz(r2), ti.x, ti.y, xi.w, h ? C.w : C.z, h ? Nj.y : Nj.x,
                                    h ? Nj.w : Nj.z, band.rc);
        if (!(fabsf(hv.x) < 1e20f && fabsf(hv.y) < 1e20f)) atomicOr(status, 4);
        atomicAdd((unsigned long long*)&nb.ihx[warp][slot], (unsigned long long)to_fixed(hv.x, (float)kScaleH));
        atomicAdd((unsigned long long*)&nb.jhx[2 * pr + h][jj], (unsigned long long)to_fixed(hv.y, (float)kScaleH));
    }
    __syncwarp();
}

// born_tile with the closed forms queued (weight 0 in the loop)
template <bool MASKED, bool CUT>
__device__ __forceinline__ void born_tile_q(const BoJs* sjg, int pr, int lane, int warp, const BoI2 (&I)[2],
                                            float2 (&ah)[2], float2& jh, const uint32_t (&sk)[2][2],
                                            const PairBand& band, BoNear& nb, int& nq, int* status) {
    const BoJs& sj = sjg[pr];
    const int src = (lane + 1) & 31;
    const float skr2 = band.skr2;
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll 2
    for (int k = 0; k < kTileJ; ++k) {
        const float4 A = sj.a[lane + k], B = sj.b[lane + k], C = sj.c[lane + k];
        const float2 s2j = make_float2(B.z, B.w), s3j = make_float2(C.x, C.y);
        float2 r2[2], hi[2], hj[2], wt[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float2 dx = __fadd2_rn(I[u].x, make_float2(A.x, A.y));
            const float2 dy = __fadd2_rn(I[u].y, make_float2(A.z, A.w));
            const float2 dz = __fadd2_rn(I[u].z, make_float2(B.x, B.y));
            r2[u] = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            if (MASKED) { // skipped pairs stay off the closed-form queue
                const int jj = (lane + k) & (kTileJ - 1);
                r2[u].x = ((sk[u][0] >> jj) & 1u) ? skr2 : r2[u].x;
                r2[u].y = ((sk[u][1] >> jj) & 1u) ? skr2 : r2[u].y;
            }
            const float2 rinv2 = make_float2(rcp_ftz(r2[u].x), rcp_ftz(r2[u].y));
            wt[u] = __fmul2_rn(rinv2, rinv2); // r^-4, the weight of both far terms
            hi[u] = __fmul2_rn(hct_series_h(__fmul2_rn(s2j, rinv2)), s3j);
            hj[u] = __fmul2_rn(hct_series_h(__fmul2_rn(I[u].s2, rinv2)), I[u].s3);
            if (CUT) { // beyond rc + s_max nothing descreens
                wt[u].x = r2[u].x >= band.rout2 ? 0.f : wt[u].x;
                wt[u].y = r2[u].y >= band.rout2 ? 0.f : wt[u].y;
            }
        }
        const uint32_t nm = (band_near<CUT>(r2[0].x, band) ? 1u : 0u) | (band_near<CUT>(r2[0].y, band) ? 2u : 0u) |
                            (band_near<CUT>(r2[1].x, band) ? 4u : 0u) | (band_near<CUT>(r2[1].y, band) ? 8u : 0u);
        if (__any_sync(0xffffffffu, nm != 0u)) {
            const uint32_t jj = (uint32_t)((lane + k) & (kTileJ - 1));
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool f = (nm >> b) & 1u;
                const uint32_t bal = __ballot_sync(0xffffffffu, f);
                if (f)
                    nb.q[warp][nq + __popc(bal & lt)] =
                        (uint32_t)lane | ((uint32_t)(b >> 1) << 5) | (jj << 6) | ((uint32_t)(b & 1) << 11) |
                        ((uint32_t)pr << 12);
                nq += __popc(bal);
            }
            // queued pairs leave the loop's sums (values too: a far form at
            // tiny r may overflow, and inf * 0 would not vanish)
            wt[0].x = (nm & 1u) ? 0.f : wt[0].x;
            wt[0].y = (nm & 2u) ? 0.f : wt[0].y;
            wt[1].x = (nm & 4u) ? 0.f : wt[1].x;
            wt[1].y = (nm & 8u) ? 0.f : wt[1].y;
            hi[0].x = (nm & 1u) ? 0.f : hi[0].x;
            hi[0].y = (nm & 2u) ? 0.f : hi[0].y;
            hi[1].x = (nm & 4u) ? 0.f : hi[1].x;
            hi[1].y = (nm & 8u) ? 0.f : hi[1].y;
            hj[0].x = (nm & 1u) ? 0.f : hj[0].x;
            hj[0].y = (nm & 2u) ? 0.f : hj[0].y;
            hj[1].x = (nm & 4u) ? 0.f : hj[1].x;
            hj[1].y = (nm & 8u) ? 0.f : hj[1].y;
            if (nq >= 64) {
                __syncwarp();
                born_flush(sjg, nb, warp, lane, nq, band, status);
                nq = 0;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (MASKED) {
                const int jj = (lane + k) & (kTileJ - 1);
                wt[u].x = ((sk[u][0] >> jj) & 1u) ? 0.f : wt[u].x;
                wt[u].y = ((sk[u][1] >> jj) & 1u) ? 0.f : wt[u].y;
            }
            ah[u] = __ffma2_rn(hi[u], wt[u], ah[u]);
            jh = __ffma2_rn(hj[u], wt[u], jh);
        }
        jh.x = __shfl_sync(0xffffffffu, jh.x, src);
        jh.y = __shfl_sync(0xffffffffu, jh.y, src);
    }
}
template <bool CUT>
__global__ void __launch_bounds__(kSymThreads, 5) k_born_sym(const SymItem* __restrict__ items, View V) {
    __shared__ BoJs sj[kSymG / 2];
    __shared__ float red[kSymG][4][kSymJ];
    __shared__ BoNear nb;
    const SymItem it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const PairBand band = pair_band(V.rfar2, V.smax32, (float)V.rgbmax);
    int ii[2];
    bool vi[2];
    BoI2 I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < N;
        const int i = vi[u] ? ii[u] : it.i0;
        const float4 xi = V.xs[A + i], pi = V.pb32[P + i];
        const float si = vi[u] ? pi.x : 0.f;
        I[u].x = splat<float2>(vi[u] ? xi.x : -kFarF);
        I[u].y = splat<float2>(vi[u] ? xi.y : -kFarF);
        I[u].z = splat<float2>(vi[u] ? xi.z : -kFarF);
        I[u].s2 = splat<float2>(si * si);
        I[u].s3 = splat<float2>(si * si * si);
        I[u].s = si;
        I[u].rt = vi[u] ? pi.y : 1.f;
        I[u].irt = vi[u] ? pi.z : 1.f;
        nb.ix[warp][u * 32 + lane] = make_float4(I[u].x.x, I[u].y.x, I[u].z.x, si);
        nb.it[warp][u * 32 + lane] = make_float2(I[u].rt, I[u].irt);
        nb.ihx[warp][u * 32 + lane] = 0;
    }
    for (int q = tid; q < kSymG * kSymJ; q += kSymThreads) nb.jhx[q / kSymJ][q % kSymJ] = 0;
    int nq = 0; // this warp's queued pairs (warp-uniform)
    long long hx[2] = {0, 0}; // i-side fixed-point sums
    int mp = V.smt_off[it.st];
    const int me = V.smt_off[it.st + 1];
    while (mp < me && V.smt_list[mp] < it.jt0) ++mp;
    int next = mp < me ? V.smt_list[mp] : 0x7fffffff;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kSymG) {
        const int ng = min(kSymG, it.jt1 - g0), npair = (ng + 1) >> 1;
        __syncthreads();
        // stage the tile pairs: thread (pair, copy, entry) writes whole rows
        for (int q = tid; q < npair * 2 * kSymJ; q += kSymThreads) {
            const int pr = q >> 6, cpy = (q >> 5) & 1, e = q & 31;
            {
                float v[2][6];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int g = 2 * pr + h, j = (g0 + g) * kSymJ + e;
                    if (g < ng && j < N) {
                        const float4 xj = V.xs[A + j], pj = V.pb32[P + j];
                        v[h][0] = -xj.x; v[h][1] = -xj.y; v[h][2] = -xj.z;
                        v[h][3] = pj.x; v[h][4] = pj.y; v[h][5] = pj.z;
                    } else { // padding: far away, no sphere
                        v[h][0] = -kFarF; v[h][1] = -kFarF; v[h][2] = -kFarF;
                        v[h][3] = 0.f; v[h][4] = 1.f; v[h][5] = 1.f;
                    }
                }
                BoJs& S = sj[pr];
                const int r = e + cpy * kSymJ;
                const float s2a = v[0][3] * v[0][3], s2b = v[1][3] * v[1][3];
                S.a[r] = make_float4(v[0][0], v[1][0], v[0][1], v[1][1]);
                S.b[r] = make_float4(v[0][2], v[1][2], s2a, s2b);
                S.c[r] = make_float4(s2a * v[0][3], s2b * v[1][3], v[0][3], v[1][3]);
                S.n[r] = make_float4(v[0][4], v[1][4], v[0][5], v[1][5]);
            }
        }
        __syncthreads();
        const int pr0 = first_live_pair(it.i0, warp, N, g0, npair);
        for (int pr = 0; pr < pr0; ++pr) {
            red[2 * pr][warp][lane] = 0.f;
            red[2 * pr + 1][warp][lane] = 0.f;
        }
        while (next < min(g0 + 2 * pr0, it.jt1)) { // masked tiles passed by
            ++mp;
            next = mp < me ? V.smt_list[mp] : 0x7fffffff;
        }
        for (int pr = pr0; pr < npair; ++pr) {
            const int jtA = g0 + 2 * pr;
            float2 jh = make_float2(0.f, 0.f);
            float2 ah[2] = {{0.f, 0.f}, {0.f, 0.f}};
            uint32_t sk[2][2] = {{0u, 0u}, {0u, 0u}};
            bool masked = false;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jt = jtA + h;
                if (jt < it.jt1 && jt == next) {
                    ++mp;
                    next = mp < me ? V.smt_list[mp] : 0x7fffffff;
                    masked = true;
                    uint32_t nbm;
#pragma unroll
                    for (int u = 0; u < 2; ++u) sym_masks(V, P, ii[u], vi[u], jt * kSymJ, N, sk[u][h], nbm);
                }
            }
            if (masked) born_tile_q<true, CUT>(sj, pr, lane, warp, I, ah, jh, sk, band, nb, nq, V.status);
            else born_tile_q<false, CUT>(sj, pr, lane, warp, I, ah, jh, sk, band, nb, nq, V.status);
            // one conversion per tile pair (the two tiles' partials summed in FP32)
#pragma unroll
            for (int u = 0; u < 2; ++u)
                hx[u] += to_fixed(ah[u].x + ah[u].y, (float)kScaleH);
            red[2 * pr][warp][lane] = jh.x;
            red[2 * pr + 1][warp][lane] = jh.y;
        }
        if (nq > 0) { // the group's staged rows are about to be replaced
            born_flush(sj, nb, warp, lane, nq, band, V.status);
            nq = 0;
        }
        __syncthreads();
        for (int q = tid; q < ng * kSymJ; q += kSymThreads) {
            const int g = q / kSymJ, j = q % kSymJ;
            const float v = red[g][0][j] + red[g][1][j] + red[g][2][j] + red[g][3][j];
            const int jg = g0 * kSymJ + q;
            if (jg < N) {
                red_add_h(&V.Hfix[A + jg], v, V.status);
                if (nb.jhx[g][j] != 0) fix_add(&V.Hfix[A + jg], nb.jhx[g][j]);
            }
            nb.jhx[g][j] = 0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (vi[u]) fix_add(&V.Hfix[A + ii[u]], hx[u] + nb.ihx[warp][u * 32 + lane]);
}

// psi, R, dR/dpsi from the descreening sums (FP64); resets the accumulators
// for this step's pair passes and, at a walker's first atom, the walker's
// energy sums and velocity scale.
__global__ void k_fin_born(View V, int a0, int n, int zero_energy) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l;
    const int w = V.a_walker[a];
    if (V.sys_ordered[V.w_sys[w]] || !V.w_local[w]) return;
    const int li = a - V.w_off[w];
    const int P = V.sys_poff[V.w_sys[w]] + li;
    // 1/rt and 1/rho come from set-up: one FP64 division per atom (FP64
    // arithmetic is scarce on GB300)
    const double rt = V.rt[P], irho = V.irho[P];
    const double psi = 0.5 * rt * ((double)V.Hfix[a] / kScaleH);
    V.Hfix[a] = 0;
    const double th = tanh(psi * (V.alpha + psi * (-V.beta + psi * V.gamma)));
    const double R = 1.0 / (V.irt[P] - th * irho);
    V.psi[a] = psi;
    V.R[a] = R;
    V.dRdpsi[a] = R * R * (1.0 - th * th) * (V.alpha + psi * (-2.0 * V.beta + 3.0 * V.gamma * psi)) * irho;
    V.Ffix[3 * a] = 0;
    V.Ffix[3 * a + 1] = 0;
    V.Ffix[3 * a + 2] = 0;
    V.dRfix[a] = 0;
    if (li == 0) {
        if (zero_energy)
            for (int t = 0; t < kEAcc; ++t) V.eacc[w * kEAcc + t] = 0;
        V.vscale[w] = 1.0;
    }
}

} // namespace cph
