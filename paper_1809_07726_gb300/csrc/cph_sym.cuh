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
// selects the series for both directions.
#pragma once
#include "cph_device.cuh"
#include "cph_internal.h"

namespace cph {

constexpr int kSymThreads = 128;
constexpr int kSymI = 256;    // atoms per i-tile (two per thread)
constexpr int kSymJ = 32;     // atoms per j-tile
constexpr int kSymChunk = 48; // j-tiles per work item at most (default; autotuned)
constexpr int kSymG = 4;      // j-tiles staged per barrier (one atom per thread)

struct SymItem {
    int w, i0, jt0, jt1, st, pad;
};

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

// ====================================================== GB + Coulomb + LJ
struct GbI {
    float x, y, z;
    float q;   // sqrt(k) q_i
    float qc;  // sqrt(k) q_i / eps_in
    float R;   // Born radius
    float dk;  // log2(e) / (4 R_i): D log2(e) = r^2 dk_i / R_j
    float sg;  // sigma_i / 2
    float se4; // 4 sqrt(eps_i)
};

struct GbAcc {
    float x, y, z, dr;
};

template <bool MASKED, bool ENERGY>
__device__ __forceinline__ void gb_tile(const float4* sa, const float4* sb, int lane, const GbI (&I)[2],
                                        GbAcc (&a)[2], GbAcc& jacc, const uint32_t (&skip)[2],
                                        const uint32_t (&nbm)[2], float tau, float iei,
                                        KSum<float>& egb, KSum<float>& ec, KSum<float>& elj) {
#pragma unroll 2
    for (int k = 0; k < kSymJ; ++k) {
        const int jj = (lane + k) & (kSymJ - 1);
        const float4 A = sa[jj];
        const float4 B = sb[jj];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float dx = I[u].x - A.x, dy = I[u].y - A.y, dz = I[u].z - A.z;
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float g = 1.f, nb = 1.f;
            if (MASKED) {
                const bool sk = (skip[u] >> jj) & 1u;
                g = sk ? 0.f : 1.f;
                nb = ((nbm[u] >> jj) & 1u) ? 0.f : 1.f;
                r2 = sk ? 1.f : r2;
            }
            const float rinv = rsqrt_ftz(r2);
            const float rinv2 = rinv * rinv;
            const float qq = I[u].q * A.w;
            const float D2 = r2 * (I[u].dk * B.y); // D log2(e), D = r^2 / (4 R_i R_j)
            const float e = exp2_ftz(-D2);
            const float fi = rsqrt_ftz(fmaf(I[u].R * B.x, e, r2));
            const float qf3 = (MASKED ? g * qq : qq) * fi * fi * fi;
            const float t = qf3 * e * fmaf(D2, kLn2, 1.f);
            a[u].dr = fmaf(t, B.x, a[u].dr);
            jacc.dr = fmaf(t, I[u].R, jacc.dr);
            const float sig = I[u].sg + B.z;
            const float sr2 = sig * sig * rinv2;
            const float sr6 = sr2 * sr2 * sr2;
            const float ep4 = (MASKED ? nb * I[u].se4 : I[u].se4) * B.w;
            const float cq = (MASKED ? nb * I[u].qc : I[u].qc) * A.w;
            const float fs = fmaf(cq, rinv, ep4 * sr6 * fmaf(12.f, sr6, -6.f)) * rinv2
                           - tau * qf3 * fmaf(-0.25f, e, 1.f);
            a[u].x = fmaf(fs, dx, a[u].x);
            a[u].y = fmaf(fs, dy, a[u].y);
            a[u].z = fmaf(fs, dz, a[u].z);
            jacc.x = fmaf(-fs, dx, jacc.x);
            jacc.y = fmaf(-fs, dy, jacc.y);
            jacc.z = fmaf(-fs, dz, jacc.z);
            if (ENERGY) {
                egb.add((MASKED ? g * qq : qq) * fi);
                ec.add(cq * rinv);
                elj.add(ep4 * sr6 * (sr6 - 1.f));
            }
        }
        const int src = (lane + 1) & 31;
        jacc.x = __shfl_sync(0xffffffffu, jacc.x, src);
        jacc.y = __shfl_sync(0xffffffffu, jacc.y, src);
        jacc.z = __shfl_sync(0xffffffffu, jacc.z, src);
        jacc.dr = __shfl_sync(0xffffffffu, jacc.dr, src);
    }
}

template <bool ENERGY>
__global__ void __launch_bounds__(kSymThreads, 6) k_gb_sym(const SymItem* __restrict__ items, View V) {
    __shared__ float4 sa[kSymG * kSymJ], sb[kSymG * kSymJ];
    __shared__ float red[kSymG][4][kSymJ][4];
    __shared__ long long sfx[kSymI][4]; // i-side fixed-point sums (each thread owns two rows)
    __shared__ double ered[kSymThreads / 32][3];
    const SymItem it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double cx = V.x[3 * (A + it.i0)], cy = V.x[3 * (A + it.i0) + 1], cz = V.x[3 * (A + it.i0) + 2];
    const float sqk = (float)V.sqrt_k, tau = (float)V.tau, iei = (float)V.inv_eps_in;
    int ii[2];
    bool vi[2];
    GbI I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < N;
        const int i = vi[u] ? ii[u] : it.i0;
        I[u].x = vi[u] ? (float)(V.x[3 * (A + i)] - cx) : -kFarF;
        I[u].y = vi[u] ? (float)(V.x[3 * (A + i) + 1] - cy) : -kFarF;
        I[u].z = vi[u] ? (float)(V.x[3 * (A + i) + 2] - cz) : -kFarF;
        I[u].q = vi[u] ? (float)(V.q[A + i] * V.sqrt_k) : 0.f;
        I[u].qc = vi[u] ? (float)(V.q[A + i] * V.sqrt_k * V.inv_eps_in) : 0.f;
        I[u].R = vi[u] ? (float)V.R[A + i] : 1.f;
        I[u].dk = vi[u] ? (float)(0.25 * 1.4426950408889634 / V.R[A + i]) : 1.f;
        I[u].sg = vi[u] ? (float)V.sigh[P + i] : 0.f;
        I[u].se4 = vi[u] ? (float)(4.0 * V.sqe[P + i]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) sfx[warp * 64 + u * 32 + lane][c] = 0;
    KSum<float> egb, ec, elj;
    int mp = V.smt_off[it.st];
    const int me = V.smt_off[it.st + 1];
    while (mp < me && V.smt_list[mp] < it.jt0) ++mp;
    int next = mp < me ? V.smt_list[mp] : 0x7fffffff;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kSymG) {
        const int ng = min(kSymG, it.jt1 - g0);
        __syncthreads();
        if (tid < ng * kSymJ) { // stage up to four j-tiles, one atom per thread
            const int j = g0 * kSymJ + tid;
            float4 a, b;
            if (j < N) {
                a = make_float4((float)(V.x[3 * (A + j)] - cx), (float)(V.x[3 * (A + j) + 1] - cy),
                                (float)(V.x[3 * (A + j) + 2] - cz), (float)V.q[A + j] * sqk);
                b = make_float4((float)V.R[A + j], (float)(1.0 / V.R[A + j]), (float)V.sigh[P + j],
                                (float)V.sqe[P + j]);
            } else {
                a = make_float4(kFarF, kFarF, kFarF, 0.f);
                b = make_float4(1.f, 1.f, 0.f, 0.f);
            }
            sa[tid] = a;
            sb[tid] = b;
        }
        __syncthreads();
        for (int g = 0; g < ng; ++g) {
            const int jt = g0 + g, j0 = jt * kSymJ;
            GbAcc jacc = {0.f, 0.f, 0.f, 0.f};
            GbAcc acc[2] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            uint32_t skip[2] = {0u, 0u}, nbm[2] = {0u, 0u};
            if (jt == next) {
                ++mp;
                next = mp < me ? V.smt_list[mp] : 0x7fffffff;
#pragma unroll
                for (int u = 0; u < 2; ++u) sym_masks(V, P, ii[u], vi[u], j0, N, skip[u], nbm[u]);
                gb_tile<true, ENERGY>(sa + g * kSymJ, sb + g * kSymJ, lane, I, acc, jacc, skip, nbm, tau,
                                      iei, egb, ec, elj);
            } else {
                gb_tile<false, ENERGY>(sa + g * kSymJ, sb + g * kSymJ, lane, I, acc, jacc, skip, nbm, tau,
                                       iei, egb, ec, elj);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) { // per-tile conversion: independent of the item's chunking
                long long* row = sfx[warp * 64 + u * 32 + lane];
                row[0] += to_fixed(acc[u].x, (float)kScaleE);
                row[1] += to_fixed(acc[u].y, (float)kScaleE);
                row[2] += to_fixed(acc[u].z, (float)kScaleE);
                row[3] += to_fixed(acc[u].dr, (float)kScaleE);
            }
            // lane l now holds the partials of partner l of this tile
            red[g][warp][lane][0] = jacc.x;
            red[g][warp][lane][1] = jacc.y;
            red[g][warp][lane][2] = jacc.z;
            red[g][warp][lane][3] = jacc.dr;
        }
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
            const long long* row = sfx[warp * 64 + u * 32 + lane];
            fix_add(&V.Ffix[3 * (A + ii[u])], row[0]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 1], row[1]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 2], row[2]);
            fix_add(&V.dRfix[A + ii[u]], row[3]);
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
            // GB pairs carry -tau; Coulomb already has 1/eps_in, LJ its factor 4
            const double scale = (tid == 0) ? -V.tau : 1.0;
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
    const int P = V.sys_poff[V.w_sys[w]] + (a - V.w_off[w]);
    const double q = V.q[a] * V.sqrt_k, R = V.R[a];
    const double dEdR = 0.5 * V.tau * ((double)V.dRfix[a] / kScaleE + q * q / (R * R));
    V.c[a] = dEdR * V.dRdpsi[a] * 0.5 * V.rt[P];
    if (ENERGY)
        atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 0],
                  (unsigned long long)__double2ll_rn(-0.5 * V.tau * q * q / R * kScaleE));
}

// ========================================================= chain rule
struct ChI {
    float x, y, z, c, s, rt;
};

template <bool MASKED>
__device__ __forceinline__ void chain_tile(const float4* sa, const float2* sb, int lane, const ChI (&I)[2],
                                           float (&ax)[2], float (&ay)[2], float (&az)[2], float& jx,
                                           float& jy, float& jz, const uint32_t (&skip)[2], float rfar2) {
#pragma unroll 2
    for (int k = 0; k < kSymJ; ++k) {
        const int jj = (lane + k) & (kSymJ - 1);
        const float4 A = sa[jj];
        const float2 B = sb[jj];
        float dx[2], dy[2], dz[2], r2[2], rinv[2], g[2];
        bool sk[2] = {false, false}, nr[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            dx[u] = I[u].x - A.x;
            dy[u] = I[u].y - A.y;
            dz[u] = I[u].z - A.z;
            r2[u] = fmaf(dx[u], dx[u], fmaf(dy[u], dy[u], dz[u] * dz[u]));
            if (MASKED) {
                sk[u] = (skip[u] >> jj) & 1u;
                r2[u] = sk[u] ? 1.f : r2[u];
            }
            rinv[u] = rsqrt_ftz(r2[u]);
            const float rinv2 = rinv[u] * rinv[u];
            g[u] = I[u].c * hct_dr_series(rinv2, rinv[u], B.x) + A.w * hct_dr_series(rinv2, rinv[u], I[u].s);
            nr[u] = r2[u] < rfar2;
        }
        // closed forms only where some lane has a pair inside r_far (rare)
        if (__any_sync(0xffffffffu, nr[0] || nr[1])) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (nr[u]) {
                    const float r = r2[u] * rinv[u];
                    g[u] = I[u].c * hct_dr(r, rinv[u], I[u].rt, B.x) + A.w * hct_dr(r, rinv[u], B.y, I[u].s);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float gg = g[u];
            if (MASKED) gg = sk[u] ? 0.f : gg;
            const float t = -gg * rinv[u];
            ax[u] = fmaf(t, dx[u], ax[u]);
            ay[u] = fmaf(t, dy[u], ay[u]);
            az[u] = fmaf(t, dz[u], az[u]);
            jx = fmaf(-t, dx[u], jx);
            jy = fmaf(-t, dy[u], jy);
            jz = fmaf(-t, dz[u], jz);
        }
        const int src = (lane + 1) & 31;
        jx = __shfl_sync(0xffffffffu, jx, src);
        jy = __shfl_sync(0xffffffffu, jy, src);
        jz = __shfl_sync(0xffffffffu, jz, src);
    }
}

__global__ void __launch_bounds__(kSymThreads, 6) k_chain_sym(const SymItem* __restrict__ items, View V) {
    __shared__ float4 sa[kSymG * kSymJ];
    __shared__ float2 sb[kSymG * kSymJ];
    __shared__ float red[kSymG][4][kSymJ][3];
    __shared__ long long sfx[kSymI][3]; // i-side fixed-point sums (each thread owns two rows)
    const SymItem it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double cx = V.x[3 * (A + it.i0)], cy = V.x[3 * (A + it.i0) + 1], cz = V.x[3 * (A + it.i0) + 2];
    const float rfar2 = V.rfar2;
    int ii[2];
    bool vi[2];
    ChI I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < N;
        const int i = vi[u] ? ii[u] : it.i0;
        I[u].x = vi[u] ? (float)(V.x[3 * (A + i)] - cx) : -kFarF;
        I[u].y = vi[u] ? (float)(V.x[3 * (A + i) + 1] - cy) : -kFarF;
        I[u].z = vi[u] ? (float)(V.x[3 * (A + i) + 2] - cz) : -kFarF;
        I[u].c = vi[u] ? (float)V.c[A + i] : 0.f;
        I[u].s = vi[u] ? (float)V.sc[P + i] : 0.f;
        I[u].rt = vi[u] ? (float)V.rt[P + i] : 1.f;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) sfx[warp * 64 + u * 32 + lane][c] = 0;
    int mp = V.smt_off[it.st];
    const int me = V.smt_off[it.st + 1];
    while (mp < me && V.smt_list[mp] < it.jt0) ++mp;
    int next = mp < me ? V.smt_list[mp] : 0x7fffffff;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kSymG) {
        const int ng = min(kSymG, it.jt1 - g0);
        __syncthreads();
        if (tid < ng * kSymJ) { // stage up to four j-tiles, one atom per thread
            const int j = g0 * kSymJ + tid;
            float4 a;
            float2 b;
            if (j < N) {
                a = make_float4((float)(V.x[3 * (A + j)] - cx), (float)(V.x[3 * (A + j) + 1] - cy),
                                (float)(V.x[3 * (A + j) + 2] - cz), (float)V.c[A + j]);
                b = make_float2((float)V.sc[P + j], (float)V.rt[P + j]);
            } else {
                a = make_float4(kFarF, kFarF, kFarF, 0.f);
                b = make_float2(0.f, 1.f);
            }
            sa[tid] = a;
            sb[tid] = b;
        }
        __syncthreads();
        for (int g = 0; g < ng; ++g) {
            const int jt = g0 + g, j0 = jt * kSymJ;
            float ax[2] = {0.f, 0.f}, ay[2] = {0.f, 0.f}, az[2] = {0.f, 0.f};
            float jx = 0.f, jy = 0.f, jz = 0.f;
            uint32_t skip[2] = {0u, 0u};
            if (jt == next) {
                ++mp;
                next = mp < me ? V.smt_list[mp] : 0x7fffffff;
                uint32_t nbm;
#pragma unroll
                for (int u = 0; u < 2; ++u) sym_masks(V, P, ii[u], vi[u], j0, N, skip[u], nbm);
                chain_tile<true>(sa + g * kSymJ, sb + g * kSymJ, lane, I, ax, ay, az, jx, jy, jz, skip, rfar2);
            } else {
                chain_tile<false>(sa + g * kSymJ, sb + g * kSymJ, lane, I, ax, ay, az, jx, jy, jz, skip, rfar2);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                long long* row = sfx[warp * 64 + u * 32 + lane];
                row[0] += to_fixed(ax[u], (float)kScaleE);
                row[1] += to_fixed(ay[u], (float)kScaleE);
                row[2] += to_fixed(az[u], (float)kScaleE);
            }
            red[g][warp][lane][0] = jx;
            red[g][warp][lane][1] = jy;
            red[g][warp][lane][2] = jz;
        }
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
            const long long* row = sfx[warp * 64 + u * 32 + lane];
            fix_add(&V.Ffix[3 * (A + ii[u])], row[0]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 1], row[1]);
            fix_add(&V.Ffix[3 * (A + ii[u]) + 2], row[2]);
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
    const int b0 = V.sys_bond_off[s], nb = V.sys_bond_off[s + 1] - b0;
    const int a0 = V.sys_ang_off[s], na = V.sys_ang_off[s + 1] - a0;
    const int t = blockIdx.x * kBondedThreads + threadIdx.x;
    double* buf = V.tforce + V.w_tf_off[w];
    const double* x = V.x;
    double eb = 0.0, ea = 0.0;
    if (t < nb) {
        const int b = b0 + t;
        const int i = V.bond_ij[2 * b], j = V.bond_ij[2 * b + 1];
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = x[3 * (A + i) + c] - x[3 * (A + j) + c];
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double dr = r - V.bond_r0[b];
        const double g = 2.0 * V.bond_k[b] * dr / r;
        for (int c = 0; c < 3; ++c) {
            buf[6 * t + c] = -g * d[c];
            buf[6 * t + 3 + c] = g * d[c];
        }
        eb = V.bond_k[b] * dr * dr;
    } else if (t < nb + na) {
        const int la = t - nb, a = a0 + la;
        const int ia = V.ang_ijk[3 * a], ib = V.ang_ijk[3 * a + 1], ic = V.ang_ijk[3 * a + 2];
        double u[3], v[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = x[3 * (A + ia) + c] - x[3 * (A + ib) + c];
            v[c] = x[3 * (A + ic) + c] - x[3 * (A + ib) + c];
        }
        const double ru = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double rv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (ru * rv);
        cs = fmin(1.0, fmax(-1.0, cs));
        const double th = acos(cs);
        const double dth = th - V.ang_t0[a];
        const double k = -2.0 * V.ang_k[a] * dth / sqrt(fmax(1e-300, 1.0 - cs * cs)); // dE/dcos
        double* o = buf + 6 * (size_t)nb + 9 * (size_t)la;
        for (int c = 0; c < 3; ++c) {
            const double gi = k * (v[c] / (ru * rv) - cs * u[c] / (ru * ru));
            const double gk = k * (u[c] / (ru * rv) - cs * v[c] / (rv * rv));
            o[c] = -gi;
            o[3 + c] = gi + gk;
            o[6 + c] = -gk;
        }
        ea = V.ang_k[a] * dth * dth;
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
    const int A = V.w_off[w], li = a - A, P = V.sys_poff[s];
    double F[3] = {(double)V.Ffix[3 * a] / kScaleE, (double)V.Ffix[3 * a + 1] / kScaleE,
                   (double)V.Ffix[3 * a + 2] / kScaleE};
    const double* buf = V.tforce + V.w_tf_off[w];
    const int b0 = V.sys_bond_off[s], nb = V.sys_bond_off[s + 1] - b0, an0 = V.sys_ang_off[s];
    for (int e = V.bond_off[P + li]; e < V.bond_off[P + li + 1]; ++e) {
        const int b = V.bond_idx[e];
        const int role = (V.bond_ij[2 * b] == li) ? 0 : 1;
        const double* o = buf + 6 * (b - b0) + 3 * role;
        for (int c = 0; c < 3; ++c) F[c] += o[c];
    }
    for (int e = V.ang_off[P + li]; e < V.ang_off[P + li + 1]; ++e) {
        const int ag = V.ang_idx[e];
        const int role = (V.ang_ijk[3 * ag] == li) ? 0 : ((V.ang_ijk[3 * ag + 1] == li) ? 1 : 2);
        const double* o = buf + 6 * (size_t)nb + 9 * (size_t)(ag - an0) + 3 * role;
        for (int c = 0; c < 3; ++c) F[c] += o[c];
    }
    V.F[3 * a] = F[0];
    V.F[3 * a + 1] = F[1];
    V.F[3 * a + 2] = F[2];
    if (!(isfinite(F[0]) && isfinite(F[1]) && isfinite(F[2]))) atomicOr(V.status, 1);
}

// ========================================================= Born radii
// Each unordered pair yields both descreening integrals, H(r, rt_i, s_j) for
// psi_i and H(r, rt_j, s_i) for psi_j (one shared distance).  Sums go to the
// int64 accumulator Hfix (scale 2^40); k_fin_born turns them into R.
struct BoI {
    float x, y, z, s, rt, irt;
};

template <bool MASKED>
__device__ __forceinline__ void born_tile(const float4* sa, const float2* sb, int lane, const BoI (&I)[2],
                                          float (&ah)[2], float& jh, const uint32_t (&skip)[2], float rfar2) {
#pragma unroll 2
    for (int k = 0; k < kSymJ; ++k) {
        const int jj = (lane + k) & (kSymJ - 1);
        const float4 A = sa[jj];
        const float2 B = sb[jj];
        float r2[2], rinv[2], hi[2], hj[2];
        bool sk[2] = {false, false}, nr[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float dx = I[u].x - A.x, dy = I[u].y - A.y, dz = I[u].z - A.z;
            r2[u] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (MASKED) {
                sk[u] = (skip[u] >> jj) & 1u;
                r2[u] = sk[u] ? 1.f : r2[u];
            }
            rinv[u] = rsqrt_ftz(r2[u]);
            hi[u] = hct_series(rinv[u], B.x);
            hj[u] = hct_series(rinv[u], I[u].s);
            nr[u] = r2[u] < rfar2;
        }
        // closed forms only where some lane has a pair inside r_far (rare)
        if (__any_sync(0xffffffffu, nr[0] || nr[1])) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (nr[u]) {
                    const float r = r2[u] * rinv[u];
                    hi[u] = hct(r, rinv[u], I[u].rt, I[u].irt, B.x);
                    hj[u] = hct(r, rinv[u], A.w, B.y, I[u].s);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (MASKED) {
                hi[u] = sk[u] ? 0.f : hi[u];
                hj[u] = sk[u] ? 0.f : hj[u];
            }
            ah[u] += hi[u];
            jh += hj[u];
        }
        jh = __shfl_sync(0xffffffffu, jh, (lane + 1) & 31);
    }
}

__global__ void __launch_bounds__(kSymThreads, 8) k_born_sym(const SymItem* __restrict__ items, View V) {
    __shared__ float4 sa[kSymG * kSymJ];
    __shared__ float2 sb[kSymG * kSymJ];
    __shared__ float red[kSymG][4][kSymJ];
    const SymItem it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double cx = V.x[3 * (A + it.i0)], cy = V.x[3 * (A + it.i0) + 1], cz = V.x[3 * (A + it.i0) + 2];
    const float rfar2 = V.rfar2;
    int ii[2];
    bool vi[2];
    BoI I[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        ii[u] = it.i0 + warp * 64 + u * 32 + lane;
        vi[u] = ii[u] < N;
        const int i = vi[u] ? ii[u] : it.i0;
        I[u].x = vi[u] ? (float)(V.x[3 * (A + i)] - cx) : -kFarF;
        I[u].y = vi[u] ? (float)(V.x[3 * (A + i) + 1] - cy) : -kFarF;
        I[u].z = vi[u] ? (float)(V.x[3 * (A + i) + 2] - cz) : -kFarF;
        I[u].s = vi[u] ? (float)V.sc[P + i] : 0.f;
        I[u].rt = vi[u] ? (float)V.rt[P + i] : 1.f;
        I[u].irt = vi[u] ? (float)(1.0 / V.rt[P + i]) : 1.f;
    }
    long long hx[2] = {0, 0}; // i-side fixed-point sums
    int mp = V.smt_off[it.st];
    const int me = V.smt_off[it.st + 1];
    while (mp < me && V.smt_list[mp] < it.jt0) ++mp;
    int next = mp < me ? V.smt_list[mp] : 0x7fffffff;
    for (int g0 = it.jt0; g0 < it.jt1; g0 += kSymG) {
        const int ng = min(kSymG, it.jt1 - g0);
        __syncthreads();
        if (tid < ng * kSymJ) { // stage up to four j-tiles, one atom per thread
            const int j = g0 * kSymJ + tid;
            float4 a;
            float2 b;
            if (j < N) {
                a = make_float4((float)(V.x[3 * (A + j)] - cx), (float)(V.x[3 * (A + j) + 1] - cy),
                                (float)(V.x[3 * (A + j) + 2] - cz), (float)V.rt[P + j]);
                b = make_float2((float)V.sc[P + j], (float)(1.0 / V.rt[P + j]));
            } else {
                a = make_float4(kFarF, kFarF, kFarF, 1.f);
                b = make_float2(0.f, 1.f);
            }
            sa[tid] = a;
            sb[tid] = b;
        }
        __syncthreads();
        for (int g = 0; g < ng; ++g) {
            const int jt = g0 + g, j0 = jt * kSymJ;
            float jh = 0.f;
            float ah[2] = {0.f, 0.f};
            uint32_t skip[2] = {0u, 0u};
            if (jt == next) {
                ++mp;
                next = mp < me ? V.smt_list[mp] : 0x7fffffff;
                uint32_t nbm;
#pragma unroll
                for (int u = 0; u < 2; ++u) sym_masks(V, P, ii[u], vi[u], j0, N, skip[u], nbm);
                born_tile<true>(sa + g * kSymJ, sb + g * kSymJ, lane, I, ah, jh, skip, rfar2);
            } else {
                born_tile<false>(sa + g * kSymJ, sb + g * kSymJ, lane, I, ah, jh, skip, rfar2);
            }
            hx[0] += to_fixed(ah[0], (float)kScaleH);
            hx[1] += to_fixed(ah[1], (float)kScaleH);
            red[g][warp][lane] = jh;
        }
        __syncthreads();
        if (tid < ng * kSymJ) {
            const int g = tid / kSymJ, j = tid % kSymJ;
            const float v = red[g][0][j] + red[g][1][j] + red[g][2][j] + red[g][3][j];
            const int jg = g0 * kSymJ + tid;
            if (jg < N) red_add_h(&V.Hfix[A + jg], v, V.status);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (vi[u]) fix_add(&V.Hfix[A + ii[u]], hx[u]);
}

// psi, R, dR/dpsi from the descreening sums (FP64); resets the accumulators
// for this step's pair passes and, at a walker's first atom, the walker's
// energy sums and velocity scale.
__global__ void k_fin_born(View V, int a0, int n, int zero_energy) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l;
    const int w = V.a_walker[a];
    const int li = a - V.w_off[w];
    const int P = V.sys_poff[V.w_sys[w]] + li;
    const double rt = V.rt[P], rho = V.rho[P];
    const double psi = 0.5 * rt * ((double)V.Hfix[a] / kScaleH);
    V.Hfix[a] = 0;
    const double th = tanh(psi * (V.alpha + psi * (-V.beta + psi * V.gamma)));
    const double R = 1.0 / (1.0 / rt - th / rho);
    V.psi[a] = psi;
    V.R[a] = R;
    V.dRdpsi[a] = R * R * (1.0 - th * th) * (V.alpha + psi * (-2.0 * V.beta + 3.0 * V.gamma * psi)) / rho;
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
