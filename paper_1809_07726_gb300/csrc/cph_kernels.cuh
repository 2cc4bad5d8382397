// Engine kernels: the per-step pair passes over every walker of the replica
// grid, bonded terms, Langevin integration, Monte-Carlo titration sweeps and
// replica exchanges.  Host code lives in cph_engine.cu.
//
// Work decomposition of the three ordered pair passes (FP64 mode).  One CTA of
// kTile threads owns kWarpAtoms consecutive atoms i, one warp each; the CTA
// sweeps all j of its walker in tiles of kTile staged in shared memory, lane l
// of a warp taking entries l, l + 32, l + 64, l + 96 of every tile, so every
// ordered pair (i, j) is evaluated by the warp of i.  A lane's partial sums
// are added per tile into its accumulator; the warp's accumulators are
// reduced by a fixed shuffle tree at the end, so the result of an atom does
// not depend on the launch shape (batched and per-replica launches agree bit
// for bit) and no atomics are needed.  A warp per atom spreads even a
// 160-atom walker over 40 CTAs (FP64 arithmetic is a small fraction of the
// chip's, so it must run on every SM).  Positions are made relative to the
// group's first atom in FP64 before any rounding.  With Real = float the
// per-tile partials go into int64 fixed-point accumulators (scales 2^32 and
// 2^40); with double everything is FP64.
//
// Tiles in which some atom i of the CTA meets itself or an excluded partner
// are listed per (system, i-tile) at set-up; only those run the masked loop.
#pragma once
#include "cph_device.cuh"
#include "cph_internal.h"

namespace cph {

constexpr int kTile = 128;
constexpr int kWarpAtoms = kTile / 32; // atoms i per CTA of the ordered passes, one warp each
constexpr float kFarF = 1.0e4f;

// Sum of a lane accumulator over the warp by a fixed shuffle tree; lane 0
// receives the total (the same order every time: deterministic).
template <class T>
__device__ __forceinline__ T warp_total(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the WPA warps that share one atom (warps g WPA .. g WPA + WPA - 1 of
// the CTA): warp totals, then the group's warps in index order through the
// 8-byte shared slots sh[4].  Every thread of the CTA must call it.  The
// result is exact in lane 0 of each warp for WPA = 1 and in every thread of
// the group for WPA > 1.
template <int WPA, class T>
__device__ __forceinline__ T group_total(T v, long long* sh) {
    v = warp_total(v);
    if (WPA == 1) return v;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) reinterpret_cast<T*>(sh)[warp] = v;
    __syncthreads();
    T t = 0;
    const int g0 = (warp / WPA) * WPA;
#pragma unroll
    for (int q = 0; q < WPA; ++q) t += reinterpret_cast<const T*>(sh)[g0 + q];
    __syncthreads();
    return t;
}

template <class Real>
struct alignas(sizeof(Real) * 4) J4 {
    Real x, y, z, w;
};

template <class Real>
struct alignas(sizeof(Real) * 2) J2 {
    Real x, y;
};

// Per-walker energy accumulators (fixed point 2^32): GB, Coulomb, LJ, bond, angle.
constexpr int kEAcc = 5;

template <class T>
__device__ inline T block_sum_128(T v, T* red) {
    // deterministic fixed-order reduction over 128 threads
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0) s = red[0] + red[1] + red[2] + red[3];
    return s;
}

// Build the exclusion / self masks of atom i for the j-tile starting at j0.
__device__ inline void tile_masks(const View& V, int P, int i, bool vi, int j0, uint32_t ex[4],
                                  uint32_t self[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) ex[q] = self[q] = 0u;
    if (!vi) return;
    int d = i - j0;
    if (d >= 0 && d < kTile) {
        self[d >> 5] |= 1u << (d & 31);
        ex[d >> 5] |= 1u << (d & 31);
    }
    for (int e = V.excl_off[P + i]; e < V.excl_off[P + i + 1]; ++e) {
        int dj = V.excl_j[e] - j0;
        if (dj >= 0 && dj < kTile) ex[dj >> 5] |= 1u << (dj & 31);
    }
}

// ------------------------------------------------------------- pass 1: Born radii
// psi_i = rt_i/2 sum_{j != i} H(r_ij, rt_i, s_j); R_i = 1/(1/rt_i - tanh(theta)/rho_i)
// with theta = alpha psi - beta psi^2 + gamma psi^3, finalised in FP64.
template <class Real, int WPA>
__global__ void __launch_bounds__(kTile) k_born(const Item* __restrict__ items, View V,
                                                int zero_energy) {
    using Pr = Prec<Real>;
    __shared__ J4<Real> sj[kTile];
    const Item it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    // WPA warps per atom i: the CTA holds kWarpAtoms / WPA atoms; `sub` indexes
    // the thread within its atom's group of 32 WPA threads
    const int tid = threadIdx.x, warp = tid >> 5, sub = tid - (warp / WPA) * 32 * WPA;
    const int i = it.i0 + warp / WPA;
    __shared__ long long gsh[kTile / 32];
    const bool vi = i < N;
    if (it.i0 == 0) {
        if (zero_energy && tid < kEAcc) V.eacc[w * kEAcc + tid] = 0;
        if (tid == kEAcc) V.vscale[w] = 1.0;
    }
    const double cx = V.x[3 * (A + it.i0)], cy = V.x[3 * (A + it.i0) + 1],
                 cz = V.x[3 * (A + it.i0) + 2];
    Real xi = Real(-kFarF), yi = Real(-kFarF), zi = Real(-kFarF), rti = Real(1);
    if (vi) {
        xi = Real(V.x[3 * (A + i)] - cx);
        yi = Real(V.x[3 * (A + i) + 1] - cy);
        zi = Real(V.x[3 * (A + i) + 2] - cz);
        rti = Real(V.rt[P + i]);
    }
    const Real irti = Real(1) / rti;
    const Real rc = Real(V.rgbmax); // Born-radius cutoff (INFINITY = none)
    typename Pr::Acc acc = 0;
    int mp = V.mt_off[it.st];
    const int me = V.mt_off[it.st + 1];
    int next = mp < me ? V.mt_list[mp] : 0x7fffffff;
    for (int j0 = 0, jt = 0; j0 < N; j0 += kTile, ++jt) {
        __syncthreads();
        {
            const int j = j0 + tid;
            J4<Real> v;
            if (j < N) {
                v.x = Real(V.x[3 * (A + j)] - cx);
                v.y = Real(V.x[3 * (A + j) + 1] - cy);
                v.z = Real(V.x[3 * (A + j) + 2] - cz);
                v.w = Real(V.sc[P + j]);
            } else {
                v.x = v.y = v.z = Real(kFarF);
                v.w = Real(0);
            }
            sj[tid] = v;
        }
        __syncthreads();
        Real part = 0;
        if (jt != next) {
#pragma unroll
            for (int k = sub; k < kTile; k += 32 * WPA) {
                const J4<Real> b = sj[k];
                const Real dx = xi - b.x, dy = yi - b.y, dz = zi - b.z;
                const Real r2 = dx * dx + dy * dy + dz * dz;
                const Real rinv = Pr::rsqrt(r2);
                part += hct(r2 * rinv, rinv, rti, irti, b.w, rc);
            }
        } else {
            ++mp;
            next = mp < me ? V.mt_list[mp] : 0x7fffffff;
            const int dself = i - j0;
#pragma unroll
            for (int k = sub; k < kTile; k += 32 * WPA) {
                const J4<Real> b = sj[k];
                const bool self = (k == dself);
                const Real dx = xi - b.x, dy = yi - b.y, dz = zi - b.z;
                Real r2 = dx * dx + dy * dy + dz * dz;
                r2 = self ? Real(1) : r2;
                const Real rinv = Pr::rsqrt(r2);
                const Real h = hct(r2 * rinv, rinv, rti, irti, b.w, rc);
                part += self ? Real(0) : h;
            }
        }
        Pr::add(acc, part, Real(kScaleH));
    }
    acc = group_total<WPA>(acc, gsh);
    if (vi && sub == 0) {
        const double sumH = Pr::value(acc, kScaleH);
        const double rt = V.rt[P + i], irho = V.irho[P + i]; // 1/rt, 1/rho from set-up
        const double psi = 0.5 * rt * sumH;
        const double th = tanh(psi * (V.alpha + psi * (-V.beta + psi * V.gamma)));
        const double R = 1.0 / (V.irt[P + i] - th * irho);
        V.psi[A + i] = psi;
        V.R[A + i] = R;
        V.Ffix[3 * (A + i)] = 0;
        V.Ffix[3 * (A + i) + 1] = 0;
        V.Ffix[3 * (A + i) + 2] = 0;
        V.dRfix[A + i] = 0;
        V.dRdpsi[A + i] = R * R * (1.0 - th * th) * (V.alpha + psi * (-2.0 * V.beta + 3.0 * V.gamma * psi)) * irho;
    }
}

// ------------------------------------------- pass 2: GB + Coulomb + LJ pair pass
// Owner i accumulates the direct force, dE_GB/dR_i and (optionally) its share
// of the energies; the epilogue turns dE/dR_i into c_i = dE/dR_i dR_i/dpsi_i rt_i/2.
template <class Real, bool ENERGY, int WPA>
__global__ void __launch_bounds__(kTile) k_gb(const Item* __restrict__ items, View V) {
    using Pr = Prec<Real>;
    using Acc = typename Pr::Acc;
    __shared__ J4<Real> sa[kTile];
    __shared__ J4<Real> sb[kTile];
    __shared__ long long red[4];
    const Item it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    // WPA warps per atom i: the CTA holds kWarpAtoms / WPA atoms; `sub` indexes
    // the thread within its atom's group of 32 WPA threads
    const int tid = threadIdx.x, warp = tid >> 5, sub = tid - (warp / WPA) * 32 * WPA;
    const int i = it.i0 + warp / WPA;
    __shared__ long long gsh[kTile / 32];
    const bool vi = i < N;
    const Real sqk = Real(V.sqrt_k);
    const double cx = V.x[3 * (A + it.i0)], cy = V.x[3 * (A + it.i0) + 1],
                 cz = V.x[3 * (A + it.i0) + 2];
    Real xi = Real(-kFarF), yi = Real(-kFarF), zi = Real(-kFarF);
    Real qi = 0, Ri = 1, iRi = 1, sgi = 0, sei = 0;
    if (vi) {
        xi = Real(V.x[3 * (A + i)] - cx);
        yi = Real(V.x[3 * (A + i) + 1] - cy);
        zi = Real(V.x[3 * (A + i) + 2] - cz);
        qi = Real(V.q[A + i]) * sqk;
        Ri = Real(V.R[A + i]);
        iRi = Real(1.0 / V.R[A + i]);
        sgi = Real(V.sigh[P + i]);
        sei = Real(V.sqe[P + i]);
    }
    const Real tau = Real(V.tau), iei = Real(V.inv_eps_in);
    const Real kap = Real(V.kappa), ieo = Real(V.inv_eps_out);
    const bool salt = V.kappa > 0; // pair sums then carry tau(f) and taud(f) per pair
    Acc fx = 0, fy = 0, fz = 0, adr = 0, egb = 0, ec = 0, elj = 0;
    int mp = V.mt_off[it.st];
    const int me = V.mt_off[it.st + 1];
    int next = mp < me ? V.mt_list[mp] : 0x7fffffff;
    for (int j0 = 0, jt = 0; j0 < N; j0 += kTile, ++jt) {
        __syncthreads();
        {
            const int j = j0 + tid;
            J4<Real> a, b;
            if (j < N) {
                a.x = Real(V.x[3 * (A + j)] - cx);
                a.y = Real(V.x[3 * (A + j) + 1] - cy);
                a.z = Real(V.x[3 * (A + j) + 2] - cz);
                a.w = Real(V.q[A + j]) * sqk;
                b.x = Real(V.R[A + j]);
                b.y = Real(1.0 / V.R[A + j]);
                b.z = Real(V.sigh[P + j]);
                b.w = Real(V.sqe[P + j]);
            } else {
                a.x = a.y = a.z = Real(kFarF);
                a.w = 0;
                b.x = b.y = Real(1);
                b.z = b.w = 0;
            }
            sa[tid] = a;
            sb[tid] = b;
        }
        __syncthreads();
        Real px = 0, py = 0, pz = 0, pdr = 0;
        KSum<Real> pgb, pc, plj;
        if (jt != next) {
#pragma unroll
            for (int k = sub; k < kTile; k += 32 * WPA) {
                const J4<Real> a = sa[k];
                const J4<Real> b = sb[k];
                const Real dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
                const Real r2 = dx * dx + dy * dy + dz * dz;
                const Real rinv = Pr::rsqrt(r2);
                const Real rinv2 = rinv * rinv;
                const Real qq = qi * a.w;
                const Real D = Real(0.25) * r2 * (iRi * b.y);
                const Real e = Pr::expm(D);
                const Real fi = Pr::rsqrt(r2 + (Ri * b.x) * e);
                const Real qf3 = qq * fi * fi * fi;
                Real tf = Real(1), td = Real(1);
                if (salt) {
                    const Real es = ieo * Pr::expm(kap / fi);
                    tf = iei - es;
                    td = tf - kap * es / fi;
                }
                pdr += td * qf3 * b.x * e * (Real(1) + D);
                const Real sig = sgi + b.z;
                const Real sr2 = sig * sig * rinv2;
                const Real sr6 = sr2 * sr2 * sr2;
                const Real ep = sei * b.w;
                const Real fs = iei * qq * rinv * rinv2 + Real(4) * ep * sr6 * (Real(12) * sr6 - Real(6)) * rinv2
                              - (salt ? td : tau) * qf3 * (Real(1) - Real(0.25) * e);
                px += fs * dx;
                py += fs * dy;
                pz += fs * dz;
                if (ENERGY) {
                    pgb.add(tf * qq * fi);
                    pc.add(qq * rinv);
                    plj.add(ep * sr6 * (sr6 - Real(1)));
                }
            }
        } else {
            ++mp;
            next = mp < me ? V.mt_list[mp] : 0x7fffffff;
            uint32_t mex[4], mself[4];
            tile_masks(V, P, i, vi, j0, mex, mself);
#pragma unroll
            for (int k = sub; k < kTile; k += 32 * WPA) {
                {
                    const int q4 = k >> 5, kk = k & 31;
                    const bool self = (mself[q4] >> kk) & 1u;
                    const bool ex = (mex[q4] >> kk) & 1u;
                    const J4<Real> a = sa[k];
                    const J4<Real> b = sb[k];
                    const Real dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
                    Real r2 = dx * dx + dy * dy + dz * dz;
                    r2 = self ? Real(1) : r2;
                    const Real g = self ? Real(0) : Real(1);
                    const Real nb = ex ? Real(0) : Real(1);
                    const Real rinv = Pr::rsqrt(r2);
                    const Real rinv2 = rinv * rinv;
                    const Real qq = qi * a.w;
                    const Real D = Real(0.25) * r2 * (iRi * b.y);
                    const Real e = Pr::expm(D);
                    const Real fi = Pr::rsqrt(r2 + (Ri * b.x) * e);
                    const Real qf3 = g * qq * fi * fi * fi;
                    Real tf = Real(1), td = Real(1);
                    if (salt) {
                        const Real es = ieo * Pr::expm(kap / fi);
                        tf = iei - es;
                        td = tf - kap * es / fi;
                    }
                    pdr += td * qf3 * b.x * e * (Real(1) + D);
                    const Real sig = sgi + b.z;
                    const Real sr2 = sig * sig * rinv2;
                    const Real sr6 = sr2 * sr2 * sr2;
                    const Real ep = nb * sei * b.w;
                    const Real fs = nb * iei * qq * rinv * rinv2
                                  + Real(4) * ep * sr6 * (Real(12) * sr6 - Real(6)) * rinv2
                                  - (salt ? td : tau) * qf3 * (Real(1) - Real(0.25) * e);
                    px += fs * dx;
                    py += fs * dy;
                    pz += fs * dz;
                    if (ENERGY) {
                        pgb.add(tf * g * qq * fi);
                        pc.add(nb * qq * rinv);
                        plj.add(ep * sr6 * (sr6 - Real(1)));
                    }
                }
            }
        }
        Pr::add(fx, px, Real(kScaleE));
        Pr::add(fy, py, Real(kScaleE));
        Pr::add(fz, pz, Real(kScaleE));
        Pr::add(adr, pdr, Real(kScaleE));
        if (ENERGY) {
            Pr::add(egb, pgb.value(), Real(kScaleE));
            Pr::add(ec, pc.value(), Real(kScaleE));
            Pr::add(elj, plj.value(), Real(kScaleE));
        }
    }
    fx = group_total<WPA>(fx, gsh);
    fy = group_total<WPA>(fy, gsh);
    fz = group_total<WPA>(fz, gsh);
    adr = group_total<WPA>(adr, gsh);
    if (ENERGY) {
        egb = group_total<WPA>(egb, gsh);
        ec = group_total<WPA>(ec, gsh);
        elj = group_total<WPA>(elj, gsh);
    }
    if (vi && sub == 0) {
        const double q = V.q[A + i] * V.sqrt_k;
        const double R = V.R[A + i];
        const double dEdR = 0.5 * (V.tau_pair * Pr::value(adr, kScaleE)
                                   + salt_taud(R, V.inv_eps_in, V.inv_eps_out, V.kappa) * q * q / (R * R))
                          - (V.sa_gamma != 0.0 ? 6.0 * sa_ace(V.sa_gamma, V.sa_probe, V.rho[P + i], R) / R : 0.0);
        V.c[A + i] = dEdR * V.dRdpsi[A + i] * 0.5 * V.rt[P + i];
        V.Fd[3 * (A + i)] = Pr::value(fx, kScaleE);
        V.Fd[3 * (A + i) + 1] = Pr::value(fy, kScaleE);
        V.Fd[3 * (A + i) + 2] = Pr::value(fz, kScaleE);
    }
    if (ENERGY) {
        long long e0 = 0, e1 = 0, e2 = 0;
        if (vi && sub == 0) {
            const double q = V.q[A + i] * V.sqrt_k;
            const double R = V.R[A + i];
            e0 = __double2ll_rn((-0.5 * (V.tau_pair * Pr::value(egb, kScaleE)
                                         + salt_tau(R, V.inv_eps_in, V.inv_eps_out, V.kappa) * q * q / R)
                                 + sa_ace(V.sa_gamma, V.sa_probe, V.rho[P + i], R)) * kScaleE);
            e1 = __double2ll_rn(0.5 * V.inv_eps_in * Pr::value(ec, kScaleE) * kScaleE);
            e2 = __double2ll_rn(2.0 * Pr::value(elj, kScaleE) * kScaleE);
        }
        long long t0 = block_sum_128(e0, red);
        long long t1 = block_sum_128(e1, red);
        long long t2 = block_sum_128(e2, red);
        if (tid == 0) {
            atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 0], (unsigned long long)t0);
            atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 1], (unsigned long long)t1);
            atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 2], (unsigned long long)t2);
        }
    }
}

// Bonded forces on atom i (system-local index li) and its owned energy
// shares (a bond or angle is owned by its first atom), split over the threads
// of the atom's group: thread l takes the atom's terms l, l + stride, ... of
// each kind (the caller sums the threads in a fixed order).
__device__ inline void bonded_atom(const View& V, int A, int P, int li, int lane, int stride, double F[3],
                                   double& eb, double& ea) {
    const double* x = V.x;
    for (int e = V.bond_off[P + li] + lane; e < V.bond_off[P + li + 1]; e += stride) {
        const int b = V.bond_idx[e];
        const int ia = V.bond_ij[2 * b], ib = V.bond_ij[2 * b + 1];
        const int o = (ia == li) ? ib : ia;
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = x[3 * (A + li) + c] - x[3 * (A + o) + c];
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double dr = r - V.bond_r0[b];
        const double g = 2.0 * V.bond_k[b] * dr / r; // one FP64 division per bond
        for (int c = 0; c < 3; ++c) F[c] -= g * d[c];
        if (ia == li) eb += V.bond_k[b] * dr * dr;
    }
    for (int e = V.ang_off[P + li] + lane; e < V.ang_off[P + li + 1]; e += stride) {
        const int a = V.ang_idx[e];
        const int ia = V.ang_ijk[3 * a], ib = V.ang_ijk[3 * a + 1], ic = V.ang_ijk[3 * a + 2];
        double u[3], v[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = x[3 * (A + ia) + c] - x[3 * (A + ib) + c];
            v[c] = x[3 * (A + ic) + c] - x[3 * (A + ib) + c];
        }
        const double ru2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double rv2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        // three FP64 divisions per angle (FP64 arithmetic is scarce on GB300)
        const double iuv = 1.0 / sqrt(ru2 * rv2), iru2 = 1.0 / ru2, irv2 = 1.0 / rv2;
        double cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) * iuv;
        cs = fmin(1.0, fmax(-1.0, cs));
        const double th = acos(cs);
        const double dth = th - V.ang_t0[a];
        const double k = -2.0 * V.ang_k[a] * dth / sqrt(fmax(1e-300, 1.0 - cs * cs)); // dE/dcos
        double gi[3], gk[3];
        for (int c = 0; c < 3; ++c) {
            gi[c] = k * (v[c] * iuv - cs * u[c] * iru2);
            gk[c] = k * (u[c] * iuv - cs * v[c] * irv2);
        }
        for (int c = 0; c < 3; ++c) {
            if (li == ia) F[c] -= gi[c];
            if (li == ic) F[c] -= gk[c];
            if (li == ib) F[c] += gi[c] + gk[c];
        }
        if (ia == li) ea += V.ang_k[a] * dth * dth;
    }
}

// FP32-mode bonded terms (the symmetric bonded kernel and the ordered chain
// kernel share them): FP64 only where a difference of nearly equal numbers
// decides the result (the separations, r^2 - r0^2, the dot and cross products
// behind the sine and cosine of theta - theta0), FP32 elsewhere (atan2f for
// theta - theta0), so that the few FP64 units of the chip are not the bound.
//
// One harmonic bond from its FP64 separation d = x_i - x_j: the force on i is
// -g d, on j +g d; e its energy.
__device__ __forceinline__ void bond_term32(const double (&d)[3], double r0d, double kbd, float& g, float& e) {
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float r = sqrtf((float)r2);
    const float dr = (float)(r2 - r0d * r0d) / (r + (float)r0d); // r - r0 at FP32 relative precision
    const float kb = (float)kbd;
    g = 2.f * kb * dr / r;
    e = kb * dr * dr;
}

// One harmonic angle i-j-k from u = x_i - x_j, v = x_k - x_j (FP64) and
// (cos theta0, sin theta0): the force on i is -gi, on k -gk, on j gi + gk;
// e its energy.
__device__ __forceinline__ void angle_term32(const double (&u)[3], const double (&v)[3], double2 cs0, double kad,
                                             float (&gi)[3], float (&gk)[3], float& e) {
    // |u||v| cos(theta) and |u||v| sin(theta) in FP64 (the norm of the cross
    // product by an FP32 reciprocal square root and one Newton step)
    const double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
    const double w2 = cx * cx + cy * cy + cz * cz;
    const double y = (double)rsqrtf(fmaxf((float)w2, 1e-30f));
    double wn = w2 * y;
    wn += 0.5 * (w2 - wn * wn) * y;
    // theta - theta0 = atan2(sin(theta - theta0), cos(theta - theta0))
    const float dth = atan2f((float)(wn * cs0.x - uv * cs0.y), (float)(uv * cs0.x + wn * cs0.y));
    const float ka = (float)kad;
    float uf[3], vf[3];
    for (int c = 0; c < 3; ++c) {
        uf[c] = (float)u[c];
        vf[c] = (float)v[c];
    }
    const float ru2 = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
    const float rv2 = vf[0] * vf[0] + vf[1] * vf[1] + vf[2] * vf[2];
    const float iuv = rsqrtf(ru2 * rv2);                     // 1 / (|u| |v|)
    const float cs = (float)uv * iuv, sn = fmaxf((float)wn * iuv, 1e-20f);
    const float k = -2.f * ka * dth / sn;                     // dE/dcos(theta)
    for (int c = 0; c < 3; ++c) {
        gi[c] = k * (vf[c] * iuv - cs * uf[c] / ru2);
        gk[c] = k * (uf[c] * iuv - cs * vf[c] / rv2);
    }
    e = ka * dth * dth;
}

// The FP32-mode terms of one atom (the ordered chain kernel: each atom takes
// the terms it is part of), its forces and energies summed in FP32.
__device__ inline void bonded_atom32(const View& V, int A, int P, int li, int lane, int stride, float F[3],
                                     float& eb, float& ea) {
    const double* x = V.x;
    for (int e = V.bond_off[P + li] + lane; e < V.bond_off[P + li + 1]; e += stride) {
        const int b = V.bond_idx[e];
        const int ia = V.bond_ij[2 * b], ib = V.bond_ij[2 * b + 1];
        const int o = (ia == li) ? ib : ia;
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = x[3 * (A + li) + c] - x[3 * (A + o) + c];
        float g, en;
        bond_term32(d, V.bond_r0[b], V.bond_k[b], g, en);
        for (int c = 0; c < 3; ++c) F[c] -= g * (float)d[c];
        if (ia == li) eb += en;
    }
    for (int e = V.ang_off[P + li] + lane; e < V.ang_off[P + li + 1]; e += stride) {
        const int a = V.ang_idx[e];
        const int ia = V.ang_ijk[3 * a], ib = V.ang_ijk[3 * a + 1], ic = V.ang_ijk[3 * a + 2];
        double u[3], v[3];
        for (int c = 0; c < 3; ++c) {
            u[c] = x[3 * (A + ia) + c] - x[3 * (A + ib) + c];
            v[c] = x[3 * (A + ic) + c] - x[3 * (A + ib) + c];
        }
        float gi[3], gk[3], en;
        angle_term32(u, v, V.ang_cs0[a], V.ang_k[a], gi, gk, en);
        for (int c = 0; c < 3; ++c) {
            if (li == ia) F[c] -= gi[c];
            if (li == ic) F[c] -= gk[c];
            if (li == ib) F[c] += gi[c] + gk[c];
        }
        if (ia == li) ea += en;
    }
}

// ------------------------------------------ pass 3: chain rule through Born radii
// F_i -= sum_j (c_i dH(r; rt_i, s_j)/dr + c_j dH(r; rt_j, s_i)/dr) (x_i - x_j)/r,
// then the direct pair force and the bonded terms are added: F is the total force.
template <class Real, bool ENERGY, int WPA>
__global__ void __launch_bounds__(kTile) k_chain(const Item* __restrict__ items, View V) {
    using Pr = Prec<Real>;
    using Acc = typename Pr::Acc;
    __shared__ J4<Real> sa[kTile];
    __shared__ J2<Real> sb[kTile];
    __shared__ long long red[4];
    const Item it = items[blockIdx.x];
    const int w = it.w, s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    // WPA warps per atom i: the CTA holds kWarpAtoms / WPA atoms; `sub` indexes
    // the thread within its atom's group of 32 WPA threads
    const int tid = threadIdx.x, warp = tid >> 5, sub = tid - (warp / WPA) * 32 * WPA;
    const int i = it.i0 + warp / WPA;
    __shared__ long long gsh[kTile / 32];
    const bool vi = i < N;
    const double cx = V.x[3 * (A + it.i0)], cy = V.x[3 * (A + it.i0) + 1],
                 cz = V.x[3 * (A + it.i0) + 2];
    Real xi = Real(-kFarF), yi = Real(-kFarF), zi = Real(-kFarF), ci = 0, si = 0, rti = 1;
    if (vi) {
        xi = Real(V.x[3 * (A + i)] - cx);
        yi = Real(V.x[3 * (A + i) + 1] - cy);
        zi = Real(V.x[3 * (A + i) + 2] - cz);
        ci = Real(V.c[A + i]);
        si = Real(V.sc[P + i]);
        rti = Real(V.rt[P + i]);
    }
    Acc fx = 0, fy = 0, fz = 0;
    const Real rc = Real(V.rgbmax); // Born-radius cutoff (INFINITY = none)
    int mp = V.mt_off[it.st];
    const int me = V.mt_off[it.st + 1];
    int next = mp < me ? V.mt_list[mp] : 0x7fffffff;
    for (int j0 = 0, jt = 0; j0 < N; j0 += kTile, ++jt) {
        __syncthreads();
        {
            const int j = j0 + tid;
            J4<Real> a;
            J2<Real> b;
            if (j < N) {
                a.x = Real(V.x[3 * (A + j)] - cx);
                a.y = Real(V.x[3 * (A + j) + 1] - cy);
                a.z = Real(V.x[3 * (A + j) + 2] - cz);
                a.w = Real(V.c[A + j]);
                b.x = Real(V.sc[P + j]);
                b.y = Real(V.rt[P + j]);
            } else {
                a.x = a.y = a.z = Real(kFarF);
                a.w = 0;
                b.x = 0;
                b.y = 1;
            }
            sa[tid] = a;
            sb[tid] = b;
        }
        __syncthreads();
        Real px = 0, py = 0, pz = 0;
        if (jt != next) {
#pragma unroll
            for (int k = sub; k < kTile; k += 32 * WPA) {
                const J4<Real> a = sa[k];
                const J2<Real> b = sb[k];
                const Real dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
                const Real r2 = dx * dx + dy * dy + dz * dz;
                const Real rinv = Pr::rsqrt(r2);
                const Real r = r2 * rinv;
                const Real g = ci * hct_dr(r, rinv, rti, b.x, rc) + a.w * hct_dr(r, rinv, b.y, si, rc);
                const Real t = -g * rinv;
                px += t * dx;
                py += t * dy;
                pz += t * dz;
            }
        } else {
            ++mp;
            next = mp < me ? V.mt_list[mp] : 0x7fffffff;
            const int dself = i - j0;
#pragma unroll
            for (int k = sub; k < kTile; k += 32 * WPA) {
                const J4<Real> a = sa[k];
                const J2<Real> b = sb[k];
                const bool self = (k == dself);
                const Real dx = xi - a.x, dy = yi - a.y, dz = zi - a.z;
                Real r2 = dx * dx + dy * dy + dz * dz;
                r2 = self ? Real(1) : r2;
                const Real rinv = Pr::rsqrt(r2);
                const Real r = r2 * rinv;
                const Real g = ci * hct_dr(r, rinv, rti, b.x, rc) + a.w * hct_dr(r, rinv, b.y, si, rc);
                const Real t = self ? Real(0) : -g * rinv;
                px += t * dx;
                py += t * dy;
                pz += t * dz;
            }
        }
        Pr::add(fx, px, Real(kScaleE));
        Pr::add(fy, py, Real(kScaleE));
        Pr::add(fz, pz, Real(kScaleE));
    }
    fx = group_total<WPA>(fx, gsh);
    fy = group_total<WPA>(fy, gsh);
    fz = group_total<WPA>(fz, gsh);
    double eb = 0.0, ea = 0.0;
    double Fb[3] = {0.0, 0.0, 0.0};
    // bonded terms of atom i over the group's threads, summed in a fixed order
    if constexpr (sizeof(Real) == 4) {
        float fb[3] = {0.f, 0.f, 0.f}, ebf = 0.f, eaf = 0.f;
        if (vi) bonded_atom32(V, A, P, i, sub, 32 * WPA, fb, ebf, eaf);
#pragma unroll
        for (int c = 0; c < 3; ++c) Fb[c] = (double)group_total<WPA>(fb[c], gsh);
        eb = (double)group_total<WPA>(ebf, gsh);
        ea = (double)group_total<WPA>(eaf, gsh);
    } else {
        if (vi) bonded_atom(V, A, P, i, sub, 32 * WPA, Fb, eb, ea);
#pragma unroll
        for (int c = 0; c < 3; ++c) Fb[c] = group_total<WPA>(Fb[c], gsh);
        eb = group_total<WPA>(eb, gsh);
        ea = group_total<WPA>(ea, gsh);
    }
    if (sub != 0) eb = ea = 0.0; // the group's totals, counted once
    if (vi && sub == 0) {
        double F[3] = {V.Fd[3 * (A + i)] + Pr::value(fx, kScaleE) + Fb[0],
                       V.Fd[3 * (A + i) + 1] + Pr::value(fy, kScaleE) + Fb[1],
                       V.Fd[3 * (A + i) + 2] + Pr::value(fz, kScaleE) + Fb[2]};
        V.F[3 * (A + i)] = F[0];
        V.F[3 * (A + i) + 1] = F[1];
        V.F[3 * (A + i) + 2] = F[2];
        if (!(isfinite(F[0]) && isfinite(F[1]) && isfinite(F[2]))) atomicOr(V.status, 1);
    }
    if (ENERGY) {
        long long t0 = block_sum_128(__double2ll_rn(eb * kScaleE), red);
        long long t1 = block_sum_128(__double2ll_rn(ea * kScaleE), red);
        if (tid == 0) {
            atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 3], (unsigned long long)t0);
            atomicAdd((unsigned long long*)&V.eacc[w * kEAcc + 4], (unsigned long long)t1);
        }
    }
}

// ------------------------------------------------------------ Langevin step
// v' = [(1 - g dt/2) v + dt A F/m + sqrt(2 g kB T A dt/m) z] / (1 + g dt/2),
// x' = x + dt v', with T the temperature of the walker's current slot and z
// three normals from one Philox draw (Box-Muller on words (0,1) and (2,3)).
template <class Real>
__device__ inline void normals3(uint64_t seed, uint32_t idx, uint32_t stream, uint64_t step,
                                Real z[3]);

template <>
__device__ inline void normals3<double>(uint64_t seed, uint32_t idx, uint32_t stream,
                                        uint64_t step, double z[3]) {
    U4 u = draw(seed, idx, stream, step, kRngLangevin);
    const double r0 = sqrt(-2.0 * log(unit_open(u.a)));
    const double r1 = sqrt(-2.0 * log(unit_open(u.c)));
    double sn, cs;
    sincospi(2.0 * unit_open(u.b), &sn, &cs);
    z[0] = r0 * cs;
    z[1] = r0 * sn;
    z[2] = r1 * cospi(2.0 * unit_open(u.d));
}

template <>
__device__ inline void normals3<float>(uint64_t seed, uint32_t idx, uint32_t stream,
                                       uint64_t step, float z[3]) {
    U4 u = draw(seed, idx, stream, step, kRngLangevin);
    const float r0 = sqrtf(-2.0f * logf((float)unit_open(u.a)));
    const float r1 = sqrtf(-2.0f * logf((float)unit_open(u.c)));
    float sn, cs;
    sincospif(2.0f * (float)unit_open(u.b), &sn, &cs);
    z[0] = r0 * cs;
    z[1] = r0 * sn;
    z[2] = r1 * cospif(2.0f * (float)unit_open(u.d));
}

template <class Real>
__global__ void k_langevin(View V, int s_off, int a0, int n) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int a = a0 + l;
    const int w = V.a_walker[a];
    if (!V.w_local[w]) return;
    const int li = a - V.w_off[w];
    const int P = V.sys_poff[V.w_sys[w]];
    const uint64_t t = (uint64_t)(*V.step + s_off);
    const int slot = V.slot_of[w];
    Real z[3];
    normals3<Real>(V.seed, (uint32_t)li, (uint32_t)w, t, z);
    // per-atom factors dt A / m and sqrt(2 g kB A dt / m), and sqrt(T) per
    // slot, are set up once: no FP64 division or square root per step
    const double sd = V.lg_sqT[slot / (V.nE * V.npH)] * V.lg_sf[P + li];
    const double im = V.lg_im[P + li], c1 = V.lg_c1, c2 = V.lg_c2;
    const double vs = V.vscale[w];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double vn = (c1 * (V.v[3 * a + c] * vs) + im * V.F[3 * a + c] + sd * (double)z[c]) * c2;
        V.v[3 * a + c] = vn;
        if (V.xprev) V.xprev[3 * a + c] = V.x[3 * a + c]; // SHAKE's reference bond vectors
        const double xn = V.x[3 * a + c] + V.dt * vn;
        V.x[3 * a + c] = xn;
        ok = ok && isfinite(xn);
    }
    if (!ok) atomicOr(V.status, 2);
}

// SHAKE (Ryckaert, Ciccotti & Berendsen 1977) after the leapfrog step, one
// thread per (walker, cluster of one heavy atom and its hydrogens): each
// constraint in turn moves its two atoms along the bond vector before the
// step, in inverse proportion to their masses, until none of the cluster's
// constraints moves (|d0^2 - d^2| <= 2 tol d0^2); velocities take the
// displacement / dt.  The sweeps are bounded; a cluster that does not settle
// raises status flag 8.
constexpr int kShakeMaxH = 8, kShakeMaxIter = 1000;

__global__ void k_shake(View V, int i0, int n) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int it = i0 + l;
    const int w = V.shk_item_w[it], c = V.shk_item_c[it];
    if (!V.w_local[w]) return;
    const int A = V.w_off[w], P = V.sys_poff[V.w_sys[w]];
    const int h0 = V.shk_off[c], nh = V.shk_off[c + 1] - h0;
    int at[kShakeMaxH + 1];
    double xo[kShakeMaxH + 1][3], xn[kShakeMaxH + 1][3], x0[kShakeMaxH + 1][3], im[kShakeMaxH + 1];
    at[0] = V.shk_heavy[c];
    for (int k = 0; k < nh; ++k) at[k + 1] = V.shk_h[h0 + k];
    for (int k = 0; k <= nh; ++k) {
        const int a = A + at[k];
        im[k] = 1.0 / V.mass[P + at[k]];
        for (int d = 0; d < 3; ++d) {
            xo[k][d] = V.xprev[3 * a + d];
            xn[k][d] = x0[k][d] = V.x[3 * a + d];
        }
    }
    const double tol2 = 2.0 * V.shake_tol;
    bool done = false;
    for (int iter = 0; iter < kShakeMaxIter && !done; ++iter) {
        done = true;
        for (int k = 1; k <= nh; ++k) {
            const double d0 = V.shk_d[h0 + k - 1];
            double rij[3], rold[3], r2 = 0.0, dot = 0.0;
            for (int d = 0; d < 3; ++d) {
                rij[d] = xn[0][d] - xn[k][d];
                rold[d] = xo[0][d] - xo[k][d];
                r2 += rij[d] * rij[d];
                dot += rold[d] * rij[d];
            }
            const double diff = d0 * d0 - r2;
            if (fabs(diff) > tol2 * d0 * d0) {
                done = false;
                const double g = diff / (2.0 * dot * (im[0] + im[k]));
                for (int d = 0; d < 3; ++d) {
                    xn[0][d] += g * rold[d] * im[0];
                    xn[k][d] -= g * rold[d] * im[k];
                }
            }
        }
    }
    if (!done) atomicOr(V.status, 8);
    for (int k = 0; k <= nh; ++k) {
        const int a = A + at[k];
        for (int d = 0; d < 3; ++d) {
            V.x[3 * a + d] = xn[k][d];
            V.v[3 * a + d] += (xn[k][d] - x0[k][d]) / V.dt;
        }
    }
}

// velocities *= vscale[walker] (a stand-alone T exchange)
__global__ void k_vscale(View V) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= V.total_atoms) return;
    const double s = V.vscale[V.a_walker[a]];
    for (int c = 0; c < 3; ++c) V.v[3 * a + c] *= s;
}

__global__ void k_vscale_reset(View V) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < V.W) V.vscale[w] = 1.0;
}

__global__ void k_tick(long long* step, long long n) { *step += n; }

} // namespace cph
