// Pair-tile arithmetic shared by the engine's FP32 passes and the
// differentiable GB energy: a lane's two i atoms against partner l + k of two
// staged j-tiles (A, B) at step k, every quantity a float2 whose halves belong
// to tile A and tile B, so that fma/add/mul.rn.f32x2 cover both tiles.
#pragma once
#include "cph_device.cuh"

namespace cph {

constexpr int kTileJ = 32; // atoms per j-tile

// Far GB pairs: with D = r^2 / (4 R_i R_j) >= 18, e^-D <= 1.6e-8, so
// 1/f = 1/r to 1e-10 relative, the GB force factor (1 - e^-D / 4) is 1 to
// 4e-9, and the pair's dE/dR term (~ e^-D (1 + D)) is below 3e-7 of its
// q_i q_j / r^3 (and far below the self and near-pair terms of dE/dR).  The
// engine's GB tiles take that form for each i-atom row of a step whose pairs
// all meet the bound (a warp vote per row), the adjoint's tiles for a step
// whose pairs all do (a warp vote per step).
constexpr float kGbFarD2 = 18.f * kLog2e; // the threshold on D log2(e)

// ========================================================= Born radii
// Each unordered pair yields both descreening integrals, H(r, rt_i, s_j) for
// psi_i (i-side sum ah) and H(r, rt_j, s_i) for psi_j (partner sum jh, which
// moves one lane per step).  In the far regime H = P(y) s^3 / r^4 with
// y = s^2 / r^2 (P the fitted series), so s^2 and s^3 are staged and 1/r^4
// serves both directions as the weight of a fused accumulate (1 for the
// closed forms, 0 for pairs that are not counted).  Bit jj of sk[u][h]
// marks a pair of i atom u and partner jj of tile h that is not counted.
struct BoI2 {
    float2 x, y, z, s2, s3; // the i atom's value in both halves
    float s, rt, irt;       // closed-form operands
};

struct BoJs {
    float4 a[2 * kTileJ]; // (-xA, -xB, -yA, -yB)
    float4 b[2 * kTileJ]; // (-zA, -zB, s2A, s2B)
    float4 c[2 * kTileJ]; // (s3A, s3B, sA, sB)
    float4 n[2 * kTileJ]; // (rtA, rtB, 1/rtA, 1/rtB): closed forms
};

// Which pairs a tile sends to the closed forms.  Without a Born-radius
// cutoff: those inside r_far.  With a cutoff rc, also the band
// rc - s_max < r < rc + s_max, where U = min(r + s, rc) may sit at rc; inside
// the band's lower edge r + s <= rc for every s, so the series still holds
// there, and beyond its upper edge every integral and derivative of the pair
// vanishes (L >= r - s_max >= rc >= U), which CUT tiles apply as a select.
// Skipped pairs take r^2 = skr2, beyond r_far and the band (results zeroed).
struct PairBand {
    float rfar2, rin2, rout2, rc, skr2;
};

// rfar2 and s_max over every atom; rc = INFINITY for no cutoff.  The band's
// edges are widened by 1e-5 so that rounding can only move a pair towards
// the closed forms.
__host__ __device__ inline PairBand pair_band(float rfar2, float smax, float rc) {
    PairBand b;
    b.rfar2 = rfar2;
    b.rc = rc;
    if (rc < INFINITY) {
        const float rin = fmaxf(rc - smax, 0.f) * (1.f - 1e-5f), rout = (rc + smax) * (1.f + 1e-5f);
        b.rin2 = rin * rin;
        b.rout2 = rout * rout;
        b.skr2 = 4.f * fmaxf(rfar2, b.rout2) + 1.f;
    } else {
        b.rin2 = b.rout2 = INFINITY;
        b.skr2 = 4.f * rfar2 + 1.f;
    }
    return b;
}

template <bool CUT>
__device__ __forceinline__ bool band_near(float r2, const PairBand& b) {
    return CUT ? (r2 < b.rfar2 || (r2 > b.rin2 && r2 < b.rout2)) : r2 < b.rfar2;
}

// Closed-form integrals of one pair inside r_far (or in the cutoff band),
// kept out of line: a warp only gets here when one of its lanes has such a
// pair, and a single copy of this code keeps the unrolled tile loops small
// enough for the instruction cache.  Returns (H(r, rt_i, s_j), H(r, rt_j, s_i)).
static __device__ __noinline__ float2 born_near(float r2, float rinv, float rt_i, float irt_i, float s_i, float s_j,
                                         float rt_j, float irt_j, float rc) {
    const float r = r2 * rinv;
    return make_float2(hct(r, rinv, rt_i, irt_i, s_j, rc), hct(r, rinv, rt_j, irt_j, s_i, rc));
}

template <bool MASKED, bool CUT>
__device__ __forceinline__ void born_tile(const BoJs& sj, int lane, const BoI2 (&I)[2], float2 (&ah)[2],
                                          float2& jh, const uint32_t (&sk)[2][2], const PairBand& band) {
    const int src = (lane + 1) & 31;
    const float skr2 = band.skr2;
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
            if (MASKED) { // skipped pairs stay off the closed-form branch
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
        // closed forms only where some lane has such a pair (rare)
        const bool nr = band_near<CUT>(r2[0].x, band) || band_near<CUT>(r2[0].y, band) ||
                        band_near<CUT>(r2[1].x, band) || band_near<CUT>(r2[1].y, band);
        if (__any_sync(0xffffffffu, nr)) {
            const float4 Nj = sj.n[lane + k];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (band_near<CUT>(r2[u].x, band)) {
                    const float2 h = born_near(r2[u].x, rsqrt_ftz(r2[u].x), I[u].rt, I[u].irt, I[u].s, C.z, Nj.x, Nj.z,
                                               band.rc);
                    hi[u].x = h.x;
                    hj[u].x = h.y;
                    wt[u].x = 1.f;
                }
                if (band_near<CUT>(r2[u].y, band)) {
                    const float2 h = born_near(r2[u].y, rsqrt_ftz(r2[u].y), I[u].rt, I[u].irt, I[u].s, C.w, Nj.y, Nj.w,
                                               band.rc);
                    hi[u].y = h.x;
                    hj[u].y = h.y;
                    wt[u].y = 1.f;
                }
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

} // namespace cph
