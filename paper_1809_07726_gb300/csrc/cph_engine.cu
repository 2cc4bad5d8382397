// Engine: set-up, Monte-Carlo titration, replica exchange and the C ABI of
// cphremd.h.  The pair passes and the integrator are in cph_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cph_kernels.cuh"
#include "cph_sym.cuh"

namespace cph {

// =====================================================================
// Monte-Carlo titration sweep
// =====================================================================
// For the visited site with charges q -> q + dq (dq only on the site's atoms),
//   dU = sum_m dq_m (A q)_m + 1/2 sum_{m,n} dq_m dq_n A_mn,
// A_ij = k/(eps_in r_ij) [not excluded] - tau k / f_ij (i != j), A_ii = -tau k / R_i,
// i.e. U_el(q + dq) - U_el(q) for U_el = E_coul + E_GB at fixed Born radii.
//
// A site's proposal (the state b drawn uniformly among the others, and ln u)
// depends only on the counter-based stream, never on the other sites'
// outcomes, and sites share no atoms.  So the sweep runs in two kernels:
//  - k_mc_site, one CTA per (walker, site): dU0, the change at the charges of
//    the sweep's start.  The linear term runs over all N atoms (threads split
//    j); the Coulomb part of excluded pairs is removed afterwards, and the
//    small quadratic term is summed in FP64 (threads split its pairs).
//  - k_mc_sweep, one CTA per walker: the sites in index order; the site's dU
//    is dU0 plus dq^T A dq' for every site of this sweep accepted before it
//    (dq' its accepted change), then the Metropolis test.
// Both sums run in fixed orders, so the result does not depend on the launch
// form.
constexpr int kMcThreads = 256;
constexpr int kMaxSiteAtoms = 64;

// A_mn * k (both i != j), without the Coulomb part when `excluded`
template <class Real>
__device__ __forceinline__ Real mc_pair(Real dx, Real dy, Real dz, Real Rm, Real Rn, bool excluded, Real iei,
                                        Real tau, Real kap, Real ieo, bool salt) {
    using Pr = Prec<Real>;
    const Real r2 = dx * dx + dy * dy + dz * dz;
    const Real rinv = Pr::rsqrt(r2);
    const Real D = Real(0.25) * r2 / (Rm * Rn);
    const Real fi = Pr::rsqrt(r2 + Rm * Rn * Pr::expm(D));
    const Real tf = salt ? iei - ieo * Pr::expm(kap / fi) : tau;
    return (excluded ? Real(0) : iei * rinv) - tf * fi;
}

template <class Real>
__device__ __forceinline__ Real mc_const(double d, float f) {
    if constexpr (sizeof(Real) == 4) return f;
    else return d;
}

__device__ inline bool mc_excluded(const View& V, int P, int at, int an) {
    for (int e = V.excl_off[P + at]; e < V.excl_off[P + at + 1]; ++e)
        if (V.excl_j[e] == an) return true;
    return false;
}

template <class Real>
__global__ void __launch_bounds__(kMcThreads) k_mc_site(View V, int kind, int s_off, int w_begin) {
    using Pr = Prec<Real>;
    using Acc = typename Pr::Acc;
    const int w = w_begin + blockIdx.y, k = blockIdx.x;
    if (!V.w_local[w]) return;
    const int s = V.w_sys[w], N = V.sys_n[s], A = V.w_off[w], P = V.sys_poff[s];
    const int g0 = V.sys_site_off[s], ns = V.sys_site_off[s + 1] - g0, so = V.w_site_off[w];
    if (k >= ns || V.site_kind[g0 + k] != kind) return;
    const int g = g0 + k;
    const uint64_t t = (uint64_t)(*V.step + s_off);
    const int tid = threadIdx.x;
    const uint32_t purpose = (kind == CPH_SITE_PH) ? kRngMcPh : kRngMcRedox;
    __shared__ Real mx[kMaxSiteAtoms], my[kMaxSiteAtoms], mz[kMaxSiteAtoms], mR[kMaxSiteAtoms],
        mdq[kMaxSiteAtoms];
    __shared__ int mat[kMaxSiteAtoms];
    __shared__ int sh_b;
    __shared__ long long redl[kMcThreads / 32];
    __shared__ double redd[kMcThreads / 32];
    const double cx = V.x[3 * A], cy = V.x[3 * A + 1], cz = V.x[3 * A + 2];
    // FP32: the host-rounded copies (no double -> float conversion in the loops)
    const Real sqk = mc_const<Real>(V.sqrt_k, V.sqk32), tau = mc_const<Real>(V.tau, V.tau32),
               iei = mc_const<Real>(V.inv_eps_in, V.iei32);
    const Real kap = mc_const<Real>(V.kappa, V.kappa32), ieo = mc_const<Real>(V.inv_eps_out, V.ieo32);
    const bool salt = V.kappa > 0;
    const int nat = V.site_nat[g], nst = V.site_nst[g], ao = V.site_aoff[g], qo = V.site_qoff[g];
    if (tid == 0) {
        const U4 u = draw(V.seed, (uint32_t)k, (uint32_t)w, t, purpose);
        const int a = V.site_state[so + k];
        const int jj = (int)floor(unit_open(u.a) * (double)(nst - 1));
        const int b = jj < a ? jj : jj + 1;
        sh_b = b;
        V.mc_from[so + k] = a;
        V.mc_to[so + k] = b;
        V.mc_lnu[so + k] = log(unit_open(u.b));
    }
    __syncthreads();
    const int b = sh_b;
    for (int m = tid; m < nat; m += kMcThreads) {
        const int at = V.site_atoms[ao + m];
        mat[m] = at;
        mx[m] = Real(V.x[3 * (A + at)] - cx);
        my[m] = Real(V.x[3 * (A + at) + 1] - cy);
        mz[m] = Real(V.x[3 * (A + at) + 2] - cz);
        mR[m] = Real(V.R[A + at]);
        mdq[m] = Real((V.site_q[qo + b * nat + m] - V.q[A + at]) * V.sqrt_k);
    }
    __syncthreads();
    Acc lin = 0;
    auto linear_j = [&](int j, Real xj, Real yj, Real zj, Real qj, Real Rj) {
        Real part = 0;
        for (int m = 0; m < nat; ++m) {
            if (mat[m] == j) {
                const Real ts = salt ? iei - ieo * Pr::expm(kap * mR[m]) : tau;
                part += mdq[m] * qj * (-ts / mR[m]);
            } else {
                part += mdq[m] * qj * mc_pair<Real>(mx[m] - xj, my[m] - yj, mz[m] - zj, mR[m], Rj, false, iei, tau,
                                                    kap, ieo, salt);
            }
        }
        Pr::add(lin, part, Real(kScaleE));
    };
    if (sizeof(Real) == 4 && !V.sys_ordered[s]) {
        // FP32 on the symmetric tiles: the partners from the step's staged FP32
        // operands (positions relative to the walker's first atom from the
        // Born-radii pass; sqrt(k) q and R staged again just before this
        // sweep), with no FP64 subtraction or conversion per partner (both
        // issue to the narrow FP64 pipe)
        for (int j = tid; j < N; j += kMcThreads) {
            const float4 p = V.xs[A + j], gj = V.gq[A + j];
            linear_j(j, Real(p.x), Real(p.y), Real(p.z), Real(gj.x), Real(gj.y));
        }
    } else {
        for (int j = tid; j < N; j += kMcThreads)
            linear_j(j, Real(V.x[3 * (A + j)] - cx), Real(V.x[3 * (A + j) + 1] - cy),
                     Real(V.x[3 * (A + j) + 2] - cz), Real(V.q[A + j]) * sqk, Real(V.R[A + j]));
    }
    // The Coulomb part of excluded pairs (index nat * nat + m) and the
    // quadratic term's pairs (index m * nat + n): in the pass's precision from
    // the site atoms' staged values (FP32: no FP64 arithmetic per pair on the
    // narrow FP64 pipe; the FP32 terms are at the linear term's accuracy), the
    // FP64 mode in FP64 from the master positions.
    double corr = 0.0;
    if (sizeof(Real) == 4) {
        const bool staged = !V.sys_ordered[s];
        for (int idx = tid; idx < nat * nat + nat; idx += kMcThreads) {
            Real term = 0;
            if (idx >= nat * nat) {
                const int m = idx - nat * nat, at = mat[m];
                for (int e = V.excl_off[P + at]; e < V.excl_off[P + at + 1]; ++e) {
                    const int j = V.excl_j[e];
                    Real xj, yj, zj, qj;
                    if (staged) {
                        const float4 p = V.xs[A + j];
                        xj = Real(p.x);
                        yj = Real(p.y);
                        zj = Real(p.z);
                        qj = Real(V.gq[A + j].x);
                    } else {
                        xj = Real(V.x[3 * (A + j)] - cx);
                        yj = Real(V.x[3 * (A + j) + 1] - cy);
                        zj = Real(V.x[3 * (A + j) + 2] - cz);
                        qj = Real(V.q[A + j]) * sqk;
                    }
                    const Real d0 = mx[m] - xj, d1 = my[m] - yj, d2 = mz[m] - zj;
                    term -= mdq[m] * qj * iei * Pr::rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
                }
            } else {
                const int m = idx / nat, n = idx % nat;
                if (n == m) {
                    const Real ts = salt ? iei - ieo * Pr::expm(kap * mR[m]) : tau;
                    term = Real(0.5) * mdq[m] * mdq[m] * (-ts / mR[m]);
                } else {
                    term = Real(0.5) * mdq[m] * mdq[n] *
                           mc_pair<Real>(mx[m] - mx[n], my[m] - my[n], mz[m] - mz[n], mR[m], mR[n],
                                         mc_excluded(V, P, mat[m], mat[n]), iei, tau, kap, ieo, salt);
                }
            }
            corr += (double)term;
        }
    } else {
        for (int idx = tid; idx < nat * nat + nat; idx += kMcThreads) {
            if (idx >= nat * nat) {
                const int m = idx - nat * nat, at = mat[m];
                const double dqm = (V.site_q[qo + b * nat + m] - V.q[A + at]);
                const double xm0 = V.x[3 * (A + at)], xm1 = V.x[3 * (A + at) + 1], xm2 = V.x[3 * (A + at) + 2];
                for (int e = V.excl_off[P + at]; e < V.excl_off[P + at + 1]; ++e) {
                    const int j = V.excl_j[e];
                    const double d0 = xm0 - V.x[3 * (A + j)], d1 = xm1 - V.x[3 * (A + j) + 1],
                                 d2 = xm2 - V.x[3 * (A + j) + 2];
                    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    corr -= dqm * V.q[A + j] * kCoulomb * V.inv_eps_in / r;
                }
                continue;
            }
            const int m = idx / nat, n = idx % nat, at = mat[m], an = mat[n];
            const double dqm = (V.site_q[qo + b * nat + m] - V.q[A + at]);
            const double dqn = (V.site_q[qo + b * nat + n] - V.q[A + an]);
            const double Rm = V.R[A + at];
            if (n == m) {
                corr += 0.5 * dqm * dqn * (-salt_tau(Rm, V.inv_eps_in, V.inv_eps_out, V.kappa) * kCoulomb / Rm);
                continue;
            }
            const double d0 = V.x[3 * (A + at)] - V.x[3 * (A + an)], d1 = V.x[3 * (A + at) + 1] - V.x[3 * (A + an) + 1],
                         d2 = V.x[3 * (A + at) + 2] - V.x[3 * (A + an) + 2];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            const double RR = Rm * V.R[A + an];
            const double f = sqrt(r2 + RR * exp(-0.25 * r2 / RR));
            double amn = -salt_tau(f, V.inv_eps_in, V.inv_eps_out, V.kappa) * kCoulomb / f;
            if (!mc_excluded(V, P, at, an)) amn += kCoulomb * V.inv_eps_in / sqrt(r2);
            corr += 0.5 * dqm * dqn * amn;
        }
    }
    // block reduction (fixed order)
    long long lv = 0;
    double tot_d = corr;
    if (sizeof(Real) == 4) lv = (long long)lin;
    else tot_d += (double)lin;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lv += __shfl_down_sync(0xffffffffu, lv, o);
        tot_d += __shfl_down_sync(0xffffffffu, tot_d, o);
    }
    if ((tid & 31) == 0) {
        redl[tid >> 5] = lv;
        redd[tid >> 5] = tot_d;
    }
    __syncthreads();
    if (tid == 0) {
        long long L = 0;
        double D = 0.0;
        for (int q = 0; q < kMcThreads / 32; ++q) {
            L += redl[q];
            D += redd[q];
        }
        V.mc_du0[so + k] = (double)L / kScaleE + D;
    }
}

template <class Real>
__global__ void __launch_bounds__(kMcThreads) k_mc_sweep(View V, int kind, int clear_others, int w_begin) {
    using Pr = Prec<Real>;
    using Acc = typename Pr::Acc;
    const int w = w_begin + blockIdx.x;
    if (!V.w_local[w]) return;
    const int s = V.w_sys[w], A = V.w_off[w], P = V.sys_poff[s];
    const int g0 = V.sys_site_off[s], ns = V.sys_site_off[s + 1] - g0, so = V.w_site_off[w];
    const int tid = threadIdx.x;
    const int slot = V.slot_of[w];
    const int iE = slot % V.nE, ipH = (slot / V.nE) % V.npH, iT = slot / (V.nE * V.npH);
    const double E = V.gE[iE], pH = V.gpH[ipH], T = V.gT[iT];
    const double kT = kBoltzmann * T;
    __shared__ Real mx[kMaxSiteAtoms], my[kMaxSiteAtoms], mz[kMaxSiteAtoms], mR[kMaxSiteAtoms],
        mdq[kMaxSiteAtoms];
    __shared__ int mat[kMaxSiteAtoms];
    __shared__ int sh_acc;
    __shared__ long long redl[kMcThreads / 32];
    __shared__ double redd[kMcThreads / 32];
    const double cx = V.x[3 * A], cy = V.x[3 * A + 1], cz = V.x[3 * A + 2];
    // FP32: the host-rounded copies (no double -> float conversion in the loops)
    const Real sqk = mc_const<Real>(V.sqrt_k, V.sqk32), tau = mc_const<Real>(V.tau, V.tau32),
               iei = mc_const<Real>(V.inv_eps_in, V.iei32);
    const Real kap = mc_const<Real>(V.kappa, V.kappa32), ieo = mc_const<Real>(V.inv_eps_out, V.ieo32);
    const bool salt = V.kappa > 0;
    int n_taken = 0; // sites of this sweep accepted so far (uniform across the CTA)
    for (int k = 0; k < ns; ++k) {
        const int g = g0 + k;
        if (V.site_kind[g] != kind) {
            if (clear_others && tid == 0) V.mc_rec[so + k].walker = -1;
            continue;
        }
        const int nat = V.site_nat[g], ao = V.site_aoff[g], qo = V.site_qoff[g], no = V.site_noff[g];
        const int a = V.mc_from[so + k], b = V.mc_to[so + k];
        Acc cross = 0;
        if (n_taken > 0) {
            __syncthreads(); // the previous site's staging is no longer read
            for (int m = tid; m < nat; m += kMcThreads) {
                const int at = V.site_atoms[ao + m];
                mat[m] = at;
                mx[m] = Real(V.x[3 * (A + at)] - cx);
                my[m] = Real(V.x[3 * (A + at) + 1] - cy);
                mz[m] = Real(V.x[3 * (A + at) + 2] - cz);
                mR[m] = Real(V.R[A + at]);
                mdq[m] = Real((V.site_q[qo + b * nat + m] - V.site_q[qo + a * nat + m]) * V.sqrt_k);
            }
            __syncthreads();
            // dq^T A dq' over the accepted earlier sites k2, pairs (m, n) split over threads
            for (int k2 = 0; k2 < k; ++k2) {
                const int g2 = g0 + k2;
                if (V.site_kind[g2] != kind || !V.mc_take[so + k2]) continue;
                const int nat2 = V.site_nat[g2], ao2 = V.site_aoff[g2], qo2 = V.site_qoff[g2];
                const int a2 = V.mc_from[so + k2], b2 = V.mc_to[so + k2];
                Real part = 0;
                for (int idx = tid; idx < nat * nat2; idx += kMcThreads) {
                    const int m = idx / nat2, n = idx % nat2;
                    const int an = V.site_atoms[ao2 + n];
                    const Real dqn = Real(V.site_q[qo2 + b2 * nat2 + n] - V.site_q[qo2 + a2 * nat2 + n]) * sqk;
                    const Real xn = Real(V.x[3 * (A + an)] - cx), yn = Real(V.x[3 * (A + an) + 1] - cy),
                               zn = Real(V.x[3 * (A + an) + 2] - cz);
                    part += mdq[m] * dqn * mc_pair<Real>(mx[m] - xn, my[m] - yn, mz[m] - zn, mR[m], Real(V.R[A + an]),
                                                         mc_excluded(V, P, mat[m], an), iei, tau, kap, ieo, salt);
                }
                Pr::add(cross, part, Real(kScaleE));
            }
        }
        long long lv = 0;
        double dv = 0.0;
        if (sizeof(Real) == 4) lv = (long long)cross;
        else dv = (double)cross;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lv += __shfl_down_sync(0xffffffffu, lv, o);
            dv += __shfl_down_sync(0xffffffffu, dv, o);
        }
        if ((tid & 31) == 0) {
            redl[tid >> 5] = lv;
            redd[tid >> 5] = dv;
        }
        __syncthreads();
        if (tid == 0) {
            long long L = 0;
            double D = 0.0;
            for (int q = 0; q < kMcThreads / 32; ++q) {
                L += redl[q];
                D += redd[q];
            }
            const double lnu = V.mc_lnu[so + k];
            const double dU = V.mc_du0[so + k] + ((double)L / kScaleE + D);
            double dG = dU - (V.site_uref[no + b] - V.site_uref[no + a]);
            if (kind == CPH_SITE_PH)
                dG += kT * kLn10 * (double)(V.site_np[no + b] - V.site_np[no + a]) * (pH - V.site_ref[g]);
            else
                dG += kFaraday * (double)(V.site_ne[no + b] - V.site_ne[no + a]) * (E - V.site_ref[g]);
            const double x = -dG / kT;
            const int acc = lnu < x ? 1 : 0;
            cph_mc_record rec;
            rec.walker = w;
            rec.site = k;
            rec.from = a;
            rec.to = b;
            rec.accepted = acc;
            rec.pad_ = 0;
            rec.dU = dU;
            rec.x = x;
            rec.lnu = lnu;
            V.mc_rec[so + k] = rec;
            V.mc_take[so + k] = acc;
            if (acc) V.site_state[so + k] = b;
            sh_acc = acc;
            const int base = (kind == CPH_SITE_PH) ? 6 : 8;
            atomicAdd((unsigned long long*)&V.stats[base], 1ull);
            if (acc) atomicAdd((unsigned long long*)&V.stats[base + 1], 1ull);
        }
        __syncthreads();
        if (sh_acc) {
            for (int m = tid; m < nat; m += kMcThreads)
                V.q[A + V.site_atoms[ao + m]] = V.site_q[qo + b * nat + m];
            ++n_taken;
        }
    }
}

// =====================================================================
// Sampling observables: one sample per walker per MD step, taken after the
// step's MC sweeps and exchange attempt.  slot_of is a permutation, so every
// (slot, site) row and every (walker, slot) cell has one writer per step:
// plain read-modify-writes, exact and in a fixed order.
// =====================================================================
constexpr int kObsThreads = 64;

// one CTA per walker, threads over its sites
__global__ void __launch_bounds__(kObsThreads) k_observe(View V) {
    const int w = blockIdx.x;
    if (!V.w_local[w]) return; // a sharded grid's counts are summed over its engines
    const int s = V.slot_of[w];
    if (threadIdx.x == 0) {
        V.visits[(long long)w * V.W + s] += 1;
        if (w == V.first_local) *V.n_obs += 1;
    }
    // the walker at slot s belongs to the system of the walker that started
    // there, so slot s's rows are laid out like walker s's sites
    const int ws0 = V.w_site_off[w], n = V.w_site_off[w + 1] - ws0;
    const long long row0 = V.w_site_off[s];
    for (int k = threadIdx.x; k < n; k += kObsThreads)
        V.occ[(row0 + k) * CPH_MAX_STATES + V.site_state[ws0 + k]] += 1;
}

// =====================================================================
// Replica exchange (one CTA): one attempt along one dimension.
// =====================================================================
__device__ inline int walker_nprot(const View& V, int w) {
    const int s = V.w_sys[w];
    int n = 0;
    for (int g = V.sys_site_off[s], k = 0; g < V.sys_site_off[s + 1]; ++g, ++k)
        n += V.site_np[V.site_noff[g] + V.site_state[V.w_site_off[w] + k]];
    return n;
}

__device__ inline int walker_nelec(const View& V, int w) {
    const int s = V.w_sys[w];
    int n = 0;
    for (int g = V.sys_site_off[s], k = 0; g < V.sys_site_off[s + 1]; ++g, ++k)
        n += V.site_ne[V.site_noff[g] + V.site_state[V.w_site_off[w] + k]];
    return n;
}

// Exchange inputs of every walker this engine advances: the total potential
// energy in fixed point (the sum of the walker's energy accumulators, exact),
// N_H and N_e of its site states, and the two sums the semi-grand T-exchange
// energy needs: sum_k U_ref,k(s_k) and sum over redox sites of N_e,k(s_k) E0_ref,k.
__global__ void k_exchange_rows(View V) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= V.W || !V.w_local[w]) return;
    long long u = 0;
    for (int t = 0; t < kEAcc; ++t) u += V.eacc[w * kEAcc + t];
    const int s = V.w_sys[w];
    int np = 0, ne = 0;
    double uref = 0.0, e0ne = 0.0;
    for (int g = V.sys_site_off[s], k = 0; g < V.sys_site_off[s + 1]; ++g, ++k) {
        const int b = V.site_state[V.w_site_off[w] + k], no = V.site_noff[g];
        np += V.site_np[no + b];
        ne += V.site_ne[no + b];
        uref += V.site_uref[no + b];
        if (V.site_kind[g] == CPH_SITE_REDOX) e0ne += (double)V.site_ne[no + b] * V.site_ref[g];
    }
    cph_exchange_row r;
    r.walker = w;
    r.n_prot = np;
    r.n_elec = ne;
    r.pad_ = 0;
    r.u_fix = u;
    r.uref_sum = uref;
    r.e0ref_ne_sum = e0ne;
    V.ex_rows[w] = r;
}

// Energy eq (5) uses for the walker of row r at redox potential E: U, or the
// semi-grand U - sum U_ref + F (N_e E - sum_redox N_e E0_ref) (CPH_TEX_SEMIGRAND).
__device__ inline double row_energy(const View& V, const cph_exchange_row& r, double E) {
    const double u = (double)r.u_fix / kScaleE;
    if (!V.tex_semigrand) return u;
    return u - r.uref_sum + kFaraday * ((double)r.n_elec * E - r.e0ref_ne_sum);
}

constexpr int kExThreads = 256;

__global__ void __launch_bounds__(kExThreads) k_exchange(View V, int dim_req, int s_off) {
    __shared__ int sdim, spar;
    const int tid = threadIdx.x;
    const uint64_t t = (uint64_t)(*V.step + s_off);
    if (tid == 0) {
        int dim = dim_req;
        if (dim < 0) {
            dim = V.order[V.ex_state[0] % V.n_order];
            V.ex_state[0] += 1;
        }
        sdim = dim;
        spar = V.ex_state[1 + dim] & 1;
        V.ex_state[1 + dim] += 1;
    }
    for (int w = tid; w < V.W; w += kExThreads) V.vscale[w] = 1.0;
    __syncthreads();
    const int dim = sdim, par = spar;
    const int nd = dim == CPH_DIM_E ? V.nE : (dim == CPH_DIM_PH ? V.npH : V.nT);
    const int nslots = V.nE * V.npH * V.nT;
    const int nlines = nslots / nd;
    const int npl = (nd - par) / 2; // pairs (m, m+1), m = par, par+2, ... , m+1 < nd
    const int total = nlines * npl;
    for (int idx = tid; idx < total; idx += kExThreads) {
        const int line = idx / npl, p = idx % npl;
        const int m = par + 2 * p;
        int s1, s2;
        if (dim == CPH_DIM_E) {
            const int ipH = line % V.npH, iT = line / V.npH;
            s1 = m + V.nE * (ipH + V.npH * iT);
            s2 = s1 + 1;
        } else if (dim == CPH_DIM_PH) {
            const int iE = line % V.nE, iT = line / V.nE;
            s1 = iE + V.nE * (m + V.npH * iT);
            s2 = s1 + V.nE;
        } else {
            const int iE = line % V.nE, ipH = line / V.nE;
            s1 = iE + V.nE * (ipH + V.npH * m);
            s2 = s1 + V.nE * V.npH;
        }
        const int w1 = V.walker_at[s1], w2 = V.walker_at[s2];
        cph_exchange_record rec;
        rec.dim = dim;
        rec.slot_lo = s1;
        rec.slot_hi = s2;
        rec.walker_lo = w1;
        rec.walker_hi = w2;
        rec.x = 0.0;
        rec.lnu = 0.0;
        if (V.w_sys[w1] != V.w_sys[w2]) {
            rec.accepted = -1;
            V.ex_rec[idx] = rec;
            continue;
        }
        const double T1 = V.gT[s1 / (V.nE * V.npH)], T2 = V.gT[s2 / (V.nE * V.npH)];
        const cph_exchange_row r1 = V.ex_rows[w1], r2 = V.ex_rows[w2];
        double x;
        if (dim == CPH_DIM_PH) {
            const double p1 = V.gpH[(s1 / V.nE) % V.npH], p2 = V.gpH[(s2 / V.nE) % V.npH];
            x = kLn10 * (p1 - p2) * (double)(r1.n_prot - r2.n_prot);
        } else if (dim == CPH_DIM_E) {
            const double e1 = V.gE[s1 % V.nE], e2 = V.gE[s2 % V.nE];
            x = kFaraday / (kBoltzmann * T1) * (e1 - e2) * (double)(r1.n_elec - r2.n_elec);
        } else { // a T line shares E: s1 and s2 have the same E index
            const double e = V.gE[s1 % V.nE];
            x = (1.0 / (kBoltzmann * T1) - 1.0 / (kBoltzmann * T2)) * (row_energy(V, r1, e) - row_energy(V, r2, e));
        }
        const U4 u = draw(V.seed, (uint32_t)s1, (uint32_t)dim, t, kRngExchange);
        const double lnu = log(unit_open(u.a));
        const int acc = lnu < x ? 1 : 0;
        rec.x = x;
        rec.lnu = lnu;
        rec.accepted = acc;
        V.ex_rec[idx] = rec;
        atomicAdd((unsigned long long*)&V.stats[2 * dim], 1ull);
        if (acc) {
            atomicAdd((unsigned long long*)&V.stats[2 * dim + 1], 1ull);
            V.walker_at[s1] = w2;
            V.walker_at[s2] = w1;
            V.slot_of[w1] = s2;
            V.slot_of[w2] = s1;
            if (dim == CPH_DIM_T) {
                V.vscale[w1] = sqrt(T2 / T1);
                V.vscale[w2] = sqrt(T1 / T2);
            }
        }
    }
    if (tid == 0) *V.ex_n = total;
}

// =====================================================================
// Set-up kernels (FP64)
// =====================================================================
// U_ref of one (site, state): U_el of the site's atoms alone in the starting
// geometry with their own Born radii.
__global__ void k_site_ref(View V, const double* __restrict__ x0, const int* __restrict__ jobs_site,
                           const int* __restrict__ jobs_state, const int* __restrict__ site_sys,
                           int n_jobs) {
    const int job = blockIdx.x * blockDim.x + threadIdx.x;
    if (job >= n_jobs) return;
    const int g = jobs_site[job], st = jobs_state[job];
    const int s = site_sys[g], P = V.sys_poff[s];
    const int nat = V.site_nat[g], ao = V.site_aoff[g], qo = V.site_qoff[g];
    double R[kMaxSiteAtoms];
    for (int m = 0; m < nat; ++m) {
        const int am = V.site_atoms[ao + m];
        const double rt = V.rt[P + am];
        double sum = 0.0;
        for (int n = 0; n < nat; ++n) {
            if (n == m) continue;
            const int an = V.site_atoms[ao + n];
            double d0 = x0[3 * (P + am)] - x0[3 * (P + an)], d1 = x0[3 * (P + am) + 1] - x0[3 * (P + an) + 1],
                   d2 = x0[3 * (P + am) + 2] - x0[3 * (P + an) + 2];
            const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            sum += hct(r, 1.0 / r, rt, 1.0 / rt, V.sc[P + an], V.rgbmax);
        }
        const double psi = 0.5 * rt * sum;
        const double th = tanh(psi * (V.alpha + psi * (-V.beta + psi * V.gamma)));
        R[m] = 1.0 / (1.0 / rt - th / V.rho[P + am]);
    }
    double U = 0.0;
    for (int m = 0; m < nat; ++m) {
        const double qm = V.site_q[qo + st * nat + m];
        U += -0.5 * salt_tau(R[m], V.inv_eps_in, V.inv_eps_out, V.kappa) * kCoulomb * qm * qm / R[m];
        const int am = V.site_atoms[ao + m];
        for (int n = m + 1; n < nat; ++n) {
            const int an = V.site_atoms[ao + n];
            const double qn = V.site_q[qo + st * nat + n];
            double d0 = x0[3 * (P + am)] - x0[3 * (P + an)], d1 = x0[3 * (P + am) + 1] - x0[3 * (P + an) + 1],
                   d2 = x0[3 * (P + am) + 2] - x0[3 * (P + an) + 2];
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            const double RR = R[m] * R[n];
            const double f = sqrt(r2 + RR * exp(-0.25 * r2 / RR));
            U += -salt_tau(f, V.inv_eps_in, V.inv_eps_out, V.kappa) * kCoulomb * qm * qn / f;
            bool ex = false;
            for (int e = V.excl_off[P + am]; e < V.excl_off[P + am + 1]; ++e)
                if (V.excl_j[e] == an) ex = true;
            if (!ex) U += kCoulomb * V.inv_eps_in * qm * qn / sqrt(r2);
        }
    }
    ((double*)V.site_uref)[V.site_noff[g] + st] = U;
}

__global__ void k_charges_from_states(View V) {
    // q of every site atom from the walker's site states
    const int w = blockIdx.x;
    const int s = V.w_sys[w], A = V.w_off[w], so = V.w_site_off[w];
    for (int g = V.sys_site_off[s], k = 0; g < V.sys_site_off[s + 1]; ++g, ++k) {
        const int st = V.site_state[so + k];
        const int nat = V.site_nat[g];
        for (int m = threadIdx.x; m < nat; m += blockDim.x)
            V.q[A + V.site_atoms[V.site_aoff[g] + m]] = V.site_q[V.site_qoff[g] + st * nat + m];
    }
}

__global__ void k_counts(View V, int* np, int* ne) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= V.W) return;
    np[w] = walker_nprot(V, w);
    ne[w] = walker_nelec(V, w);
}

} // namespace cph

// =====================================================================
// Host side
// =====================================================================
using namespace cph;

namespace {

thread_local std::string g_last_error = "no error";

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
};

} // namespace

struct cph_engine {
    std::string err = "no error";
    View V{};
    DevBuf mem;
    int precision = CPH_PREC_FP32;
    int launch_mode = 0; // 0 batched, 1 per replica
    int n_shk = 0;                  // SHAKE work items (walker, cluster); 0 when off
    std::vector<int> h_shk_w_off;   // per-walker ranges of the SHAKE items
    int mc_ph = 0, mc_redox = 0, ex_every = 0;
    long long h_step = 0;
    int n_sys = 0;
    std::vector<int> h_sys_n, h_w_sys, h_w_off, h_w_site_off, h_sys_site_off;
    std::vector<int> h_site_nst, h_site_kind, h_site_noff, h_site_np, h_site_ne;
    int n_site_states = 0;
    // ordered (one warp per atom) items: every walker in FP64 mode, the walkers
    // of the systems whose tile shape is CPH_SHAPE_WARP_PER_ATOM in FP32 mode
    Item* d_items = nullptr;
    int n_items = 0;
    std::vector<int> item_w_off; // per-walker item ranges (items grouped by walker, per-replica mode)
    Item* d_items_by_w = nullptr;
    std::vector<int> h_sys_shape;  // CPH_SHAPE_* per system (FP32 mode)
    int* d_sys_ordered = nullptr;  // 1 where a system runs the ordered passes
    int ordered_wpa = 1;           // warps per atom of the ordered passes (1 or 4)
    std::vector<int> h_w_local;    // 1 for the walkers this engine advances
    int* d_w_local = nullptr;
    bool sharded = false;          // some walker is not local
    cph_exchange_row* d_rows = nullptr;
    SymItem* d_sym = nullptr;          // symmetric FP32 items, largest system first
    SymItem* d_sym_by_w = nullptr;     // grouped by walker (per-replica mode)
    int n_sym = 0;
    int sym_chunk = kSymChunk;         // j-tiles per symmetric work item (autotuned)
    int max_sites = 0;                 // largest site count of any system
    int max_terms = 0;                 // largest bonds + angles count of any system
    std::vector<int> sym_w_off, h_sys_sst_off, h_sys_st_off;
    int ex_cap = 0;
    int mc_kinds_last = 0;
    cudaStream_t cap_stream = nullptr;
    // per-replica launches on several streams: walker w on rs[w % n_rs]
    int n_rs = 1;
    cudaStream_t rs[32] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[32] = {};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_period = 0;
    ~cph_engine() {
        for (auto& g : graph)
            if (g) cudaGraphExecDestroy(g);
        if (d_sym) cudaFree(d_sym);
        if (d_sym_by_w) cudaFree(d_sym_by_w);
        if (d_items) cudaFree(d_items);
        if (d_items_by_w) cudaFree(d_items_by_w);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (int k = 0; k < 32; ++k) {
            if (rs[k]) cudaStreamDestroy(rs[k]);
            if (ev_join[k]) cudaEventDestroy(ev_join[k]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }
};

namespace {

} // namespace

// shared with the differentiable-energy translation unit
void cph_internal_set_error(const std::string& m) { g_last_error = m; }

namespace {

int fail(cph_engine* e, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (e) e->err = buf;
    g_last_error = buf;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t ce_ = (call);                                                             \
        if (ce_ != cudaSuccess)                                                               \
            return fail(E, ce_ == cudaErrorMemoryAllocation ? CPH_E_OOM : CPH_E_CUDA,         \
                        "%s failed: %s", #call, cudaGetErrorString(ce_));                      \
    } while (0)

template <class T>
int upload(cph_engine* E, const std::vector<T>& h, T** d) {
    size_t n = std::max<size_t>(1, h.size());
    void* p = nullptr;
    CK(cudaMalloc(&p, n * sizeof(T)));
    E->mem.ptrs.push_back(p);
    if (!h.empty()) CK(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *d = (T*)p;
    return CPH_OK;
}

template <class T>
int alloc0(cph_engine* E, size_t n, T** d) {
    void* p = nullptr;
    CK(cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(T)));
    E->mem.ptrs.push_back(p);
    CK(cudaMemset(p, 0, std::max<size_t>(1, n) * sizeof(T)));
    *d = (T*)p;
    return CPH_OK;
}

#define TRY(x)                     \
    do {                           \
        int rc_ = (x);             \
        if (rc_ != CPH_OK) return rc_; \
    } while (0)

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// At most this many atoms on the FP64 ordered passes: four warps per atom.
constexpr long long kOrderedFewAtoms = 2048;

// Whether walkers of system s run the ordered passes (one warp per atom i):
// always in FP64 mode, by the system's tile shape in FP32 mode.
bool sys_ordered(const cph_engine* E, int s) {
    return E->precision == CPH_PREC_FP64 || E->h_sys_shape[s] == CPH_SHAPE_WARP_PER_ATOM;
}

// ---- launch helpers
// The ordered passes run one warp per atom (four atoms per CTA), or, in FP64
// mode with few atoms (E->ordered_wpa = 4), four warps per atom: even a single
// small walker then spreads its FP64 work over one CTA per atom.
template <class Real, int WPA>
void born_t(const Item* items, int n, View V, int ze, cudaStream_t st) {
    k_born<Real, WPA><<<n, kTile, 0, st>>>(items, V, ze);
}
template <class Real, int WPA>
void gb_t(const Item* items, int n, View V, bool energy, cudaStream_t st) {
    if (energy) k_gb<Real, true, WPA><<<n, kTile, 0, st>>>(items, V);
    else k_gb<Real, false, WPA><<<n, kTile, 0, st>>>(items, V);
}
template <class Real, int WPA>
void chain_t(const Item* items, int n, View V, bool energy, cudaStream_t st) {
    if (energy) k_chain<Real, true, WPA><<<n, kTile, 0, st>>>(items, V);
    else k_chain<Real, false, WPA><<<n, kTile, 0, st>>>(items, V);
}

int launch_born(cph_engine* E, const Item* items, int n, bool zero_energy, cudaStream_t st) {
    if (n <= 0) return CPH_OK;
    const bool f32 = E->precision == CPH_PREC_FP32, w4 = E->ordered_wpa == 4;
    const int ze = zero_energy ? 1 : 0;
    if (f32) (w4 ? born_t<float, 4> : born_t<float, 1>)(items, n, E->V, ze, st);
    else (w4 ? born_t<double, 4> : born_t<double, 1>)(items, n, E->V, ze, st);
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_gb(cph_engine* E, const Item* items, int n, bool energy, cudaStream_t st) {
    if (n <= 0) return CPH_OK;
    const bool f32 = E->precision == CPH_PREC_FP32, w4 = E->ordered_wpa == 4;
    if (f32) (w4 ? gb_t<float, 4> : gb_t<float, 1>)(items, n, E->V, energy, st);
    else (w4 ? gb_t<double, 4> : gb_t<double, 1>)(items, n, E->V, energy, st);
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_chain(cph_engine* E, const Item* items, int n, bool energy, cudaStream_t st) {
    if (n <= 0) return CPH_OK;
    const bool f32 = E->precision == CPH_PREC_FP32, w4 = E->ordered_wpa == 4;
    if (f32) (w4 ? chain_t<float, 4> : chain_t<float, 1>)(items, n, E->V, energy, st);
    else (w4 ? chain_t<double, 4> : chain_t<double, 1>)(items, n, E->V, energy, st);
    CK(cudaGetLastError());
    return CPH_OK;
}

// The three pair passes (plus bonded terms) for every walker.
int launch_forces(cph_engine* E, bool energy, cudaStream_t st, bool mc_between, int s_off,
                  int mc_kinds);

// Per-replica mode on n_rs > 1 streams: every per-walker launch sequence is
// forked from the caller's stream and joined back to it, so ordering against
// everything else on that stream (and stream capture) is kept.
int fan_out(cph_engine* E, cudaStream_t st) {
    if (E->launch_mode == 0 || E->n_rs <= 1) return CPH_OK;
    CK(cudaEventRecord(E->ev_fork, st));
    for (int k = 0; k < E->n_rs; ++k) CK(cudaStreamWaitEvent(E->rs[k], E->ev_fork, 0));
    return CPH_OK;
}

int fan_in(cph_engine* E, cudaStream_t st) {
    if (E->launch_mode == 0 || E->n_rs <= 1) return CPH_OK;
    for (int k = 0; k < E->n_rs; ++k) {
        CK(cudaEventRecord(E->ev_join[k], E->rs[k]));
        CK(cudaStreamWaitEvent(st, E->ev_join[k], 0));
    }
    return CPH_OK;
}

cudaStream_t lane_stream(const cph_engine* E, int w, cudaStream_t st) {
    return E->n_rs > 1 ? E->rs[w % E->n_rs] : st;
}

int launch_stage(cph_engine* E, int pass, int a0, int n, cudaStream_t st);

int launch_mc(cph_engine* E, int kinds, int s_off, cudaStream_t st) {
    const int W = E->V.W;
    int first = 1;
    for (int kind : {CPH_SITE_PH, CPH_SITE_REDOX}) {
        const int bit = (kind == CPH_SITE_PH) ? CPH_MC_PH : CPH_MC_REDOX;
        if (!(kinds & bit)) continue;
        if (E->max_sites <= 0) break;
        const bool f32 = E->precision == CPH_PREC_FP32;
        // the per-site kernel reads sqrt(k) q and R from the FP32 staging of the
        // symmetric tiles: stage them at this sweep's charges
        if (E->launch_mode == 0) {
            if (f32 && E->n_sym > 0) TRY(launch_stage(E, 1, 0, E->V.total_atoms, st));
            const dim3 g1(E->max_sites, W);
            if (f32) k_mc_site<float><<<g1, kMcThreads, 0, st>>>(E->V, kind, s_off, 0);
            else k_mc_site<double><<<g1, kMcThreads, 0, st>>>(E->V, kind, s_off, 0);
            if (f32) k_mc_sweep<float><<<W, kMcThreads, 0, st>>>(E->V, kind, first, 0);
            else k_mc_sweep<double><<<W, kMcThreads, 0, st>>>(E->V, kind, first, 0);
        } else {
            TRY(fan_out(E, st));
            for (int w = 0; w < W; ++w) {
                if (!E->h_w_local[w]) continue;
                cudaStream_t s = lane_stream(E, w, st);
                if (f32 && !sys_ordered(E, E->h_w_sys[w]))
                    TRY(launch_stage(E, 1, E->h_w_off[w], E->h_w_off[w + 1] - E->h_w_off[w], s));
                if (f32) k_mc_site<float><<<E->max_sites, kMcThreads, 0, s>>>(E->V, kind, s_off, w);
                else k_mc_site<double><<<E->max_sites, kMcThreads, 0, s>>>(E->V, kind, s_off, w);
                if (f32) k_mc_sweep<float><<<1, kMcThreads, 0, s>>>(E->V, kind, first, w);
                else k_mc_sweep<double><<<1, kMcThreads, 0, s>>>(E->V, kind, first, w);
            }
            TRY(fan_in(E, st));
        }
        first = 0;
        CK(cudaGetLastError());
    }
    E->mc_kinds_last = kinds;
    return CPH_OK;
}

// FP32: symmetric GB and chain passes (each unordered pair once), then the
// per-atom finishing kernels; FP64: ordered passes (bonded terms in k_chain).
int launch_sym_pair(cph_engine* E, const SymItem* items, int n, bool energy, int pass,
                    cudaStream_t st) {
    if (n <= 0) return CPH_OK;
    const bool cut = E->V.rgbmax < INFINITY;
    if (pass == 0) {
        if (cut) k_born_sym<true><<<n, kSymThreads, 0, st>>>(items, E->V);
        else k_born_sym<false><<<n, kSymThreads, 0, st>>>(items, E->V);
    } else if (pass == 2) {
        if (cut) k_chain_sym<true><<<n, kSymThreads, 0, st>>>(items, E->V);
        else k_chain_sym<false><<<n, kSymThreads, 0, st>>>(items, E->V);
    }
    else if (E->V.kappa > 0) {
        if (energy) k_gb_sym<true, true><<<n, kSymThreads, 0, st>>>(items, E->V);
        else k_gb_sym<false, true><<<n, kSymThreads, 0, st>>>(items, E->V);
    } else if (energy) k_gb_sym<true, false><<<n, kSymThreads, 0, st>>>(items, E->V);
    else k_gb_sym<false, false><<<n, kSymThreads, 0, st>>>(items, E->V);
    CK(cudaGetLastError());
    return CPH_OK;
}

// operand staging of the FP32 pair kernels: positions before the Born-radii
// pass, charge and radius terms before the GB pass (after any MC sweep)
int launch_stage(cph_engine* E, int pass, int a0, int n, cudaStream_t st) {
    const int bs = 256, g = (n + bs - 1) / bs;
    if (n <= 0 || pass == 2) return CPH_OK;
    if (pass == 0) k_stage_x<<<g, bs, 0, st>>>(E->V, a0, n);
    else k_stage_gb<<<g, bs, 0, st>>>(E->V, a0, n);
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_atoms(cph_engine* E, int which, bool energy, int a0, int n, cudaStream_t st) {
    const int bs = 256, g = (n + bs - 1) / bs;
    if (n <= 0) return CPH_OK;
    if (which == 2) {
        k_fin_born<<<g, bs, 0, st>>>(E->V, a0, n, energy ? 1 : 0);
    } else if (which == 0) {
        if (energy) k_fin_c<true><<<g, bs, 0, st>>>(E->V, a0, n);
        else k_fin_c<false><<<g, bs, 0, st>>>(E->V, a0, n);
    } else {
        k_final_forces<<<g, bs, 0, st>>>(E->V, a0, n);
    }
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_bonded(cph_engine* E, bool energy, int w0, int nw, cudaStream_t st) {
    if (E->max_terms <= 0 || nw <= 0) return CPH_OK;
    dim3 grid((E->max_terms + kBondedThreads - 1) / kBondedThreads, nw);
    if (energy) k_bonded_terms<true><<<grid, kBondedThreads, 0, st>>>(E->V, w0);
    else k_bonded_terms<false><<<grid, kBondedThreads, 0, st>>>(E->V, w0);
    CK(cudaGetLastError());
    return CPH_OK;
}

// pass: 0 born, 1 GB (+ finish), 2 chain (+ bonded terms, finish)
int launch_pass(cph_engine* E, int pass, bool energy, cudaStream_t st) {
    const bool fp32 = E->precision == CPH_PREC_FP32;
    const int W = E->V.W;
    const int fin = pass == 0 ? 2 : (pass == 1 ? 0 : 1);
    if (E->launch_mode == 0) {
        if (!fp32) {
            if (pass == 0) return launch_born(E, E->d_items, E->n_items, energy, st);
            return pass == 1 ? launch_gb(E, E->d_items, E->n_items, energy, st)
                             : launch_chain(E, E->d_items, E->n_items, energy, st);
        }
        if (E->n_sym > 0) {
            TRY(launch_stage(E, pass, 0, E->V.total_atoms, st));
            TRY(launch_sym_pair(E, E->d_sym, E->n_sym, energy, pass, st));
            if (pass == 2) TRY(launch_bonded(E, energy, 0, E->V.W, st));
            TRY(launch_atoms(E, fin, energy, 0, E->V.total_atoms, st));
        }
        if (E->n_items > 0) { // systems on the ordered passes (bonded terms in k_chain)
            if (pass == 0) TRY(launch_born(E, E->d_items, E->n_items, energy, st));
            else TRY(pass == 1 ? launch_gb(E, E->d_items, E->n_items, energy, st)
                               : launch_chain(E, E->d_items, E->n_items, energy, st));
        }
        return CPH_OK;
    }
    TRY(fan_out(E, st));
    for (int w = 0; w < W; ++w) {
        if (!E->h_w_local[w]) continue;
        const Item* it = E->d_items_by_w + E->item_w_off[w];
        const int ni = E->item_w_off[w + 1] - E->item_w_off[w];
        cudaStream_t s = lane_stream(E, w, st);
        if (!fp32 || sys_ordered(E, E->h_w_sys[w])) {
            if (pass == 0) TRY(launch_born(E, it, ni, energy, s));
            else TRY(pass == 1 ? launch_gb(E, it, ni, energy, s) : launch_chain(E, it, ni, energy, s));
        } else {
            TRY(launch_stage(E, pass, E->h_w_off[w], E->h_w_off[w + 1] - E->h_w_off[w], s));
            TRY(launch_sym_pair(E, E->d_sym_by_w + E->sym_w_off[w], E->sym_w_off[w + 1] - E->sym_w_off[w],
                                energy, pass, s));
            if (pass == 2) TRY(launch_bonded(E, energy, w, 1, s));
            TRY(launch_atoms(E, fin, energy, E->h_w_off[w], E->h_w_off[w + 1] - E->h_w_off[w], s));
        }
    }
    return fan_in(E, st);
}

int launch_forces(cph_engine* E, bool energy, cudaStream_t st, bool mc_between, int s_off,
                  int mc_kinds) {
    TRY(launch_pass(E, 0, energy, st));
    if (mc_between && mc_kinds) TRY(launch_mc(E, mc_kinds, s_off, st));
    TRY(launch_pass(E, 1, energy, st));
    TRY(launch_pass(E, 2, energy, st));
    return CPH_OK;
}

int launch_langevin(cph_engine* E, int s_off, cudaStream_t st) {
    const int bs = 256;
    auto one = [&](int a0, int n, cudaStream_t s) {
        if (E->precision == CPH_PREC_FP32)
            k_langevin<float><<<(n + bs - 1) / bs, bs, 0, s>>>(E->V, s_off, a0, n);
        else
            k_langevin<double><<<(n + bs - 1) / bs, bs, 0, s>>>(E->V, s_off, a0, n);
    };
    auto shk = [&](int i0, int n, cudaStream_t s) {
        if (n > 0) k_shake<<<(n + 127) / 128, 128, 0, s>>>(E->V, i0, n);
    };
    if (E->launch_mode == 0) {
        one(0, E->V.total_atoms, st);
        shk(0, E->n_shk, st);
    } else {
        TRY(fan_out(E, st));
        for (int w = 0; w < E->V.W; ++w) {
            if (!E->h_w_local[w]) continue;
            cudaStream_t s = lane_stream(E, w, st);
            one(E->h_w_off[w], E->h_w_off[w + 1] - E->h_w_off[w], s);
            if (E->n_shk) shk(E->h_shk_w_off[w], E->h_shk_w_off[w + 1] - E->h_shk_w_off[w], s);
        }
        TRY(fan_in(E, st));
    }
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_exchange_rows(cph_engine* E, cudaStream_t st) {
    const int bs = 128;
    k_exchange_rows<<<(E->V.W + bs - 1) / bs, bs, 0, st>>>(E->V);
    CK(cudaGetLastError());
    return CPH_OK;
}

// one exchange attempt from the rows in V.ex_rows (every walker's)
int launch_exchange_only(cph_engine* E, int dim, int s_off, cudaStream_t st) {
    k_exchange<<<1, kExThreads, 0, st>>>(E->V, dim, s_off);
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_exchange(cph_engine* E, int dim, int s_off, cudaStream_t st) {
    TRY(launch_exchange_rows(E, st));
    return launch_exchange_only(E, dim, s_off, st);
}

int launch_observe(cph_engine* E, cudaStream_t st) {
    k_observe<<<E->V.W, kObsThreads, 0, st>>>(E->V);
    CK(cudaGetLastError());
    return CPH_OK;
}

int launch_tick(cph_engine* E, long long n, cudaStream_t st) {
    k_tick<<<1, 1, 0, st>>>(E->V.step, n);
    CK(cudaGetLastError());
    return CPH_OK;
}

// Schedule of global step t (see cph_run in cphremd.h).
int enqueue_step(cph_engine* E, long long t, int s_off, bool full_schedule, cudaStream_t st) {
    int kinds = 0;
    bool exch = false;
    if (full_schedule && t > 0) {
        if (E->mc_ph > 0 && t % E->mc_ph == 0) kinds |= CPH_MC_PH;
        if (E->mc_redox > 0 && t % E->mc_redox == 0) kinds |= CPH_MC_REDOX;
        exch = E->ex_every > 0 && t % E->ex_every == 0;
    }
    TRY(launch_forces(E, exch, st, true, s_off, kinds));
    if (exch) TRY(launch_exchange(E, CPH_DIM_NEXT, s_off, st));
    TRY(launch_observe(E, st));
    TRY(launch_langevin(E, s_off, st));
    return CPH_OK;
}

long long gcdll(long long a, long long b) { return b ? gcdll(b, a % b) : a; }

int schedule_period(const cph_engine* E) {
    long long p = 1;
    for (int v : {E->mc_ph, E->mc_redox, E->ex_every})
        if (v > 0) p = p / gcdll(p, v) * v;
    return (int)std::min<long long>(p, 1 << 20);
}

int get_graph(cph_engine* E, cudaGraphExec_t* out) {
    const int mode = E->launch_mode;
    if (E->graph[mode]) {
        *out = E->graph[mode];
        return CPH_OK;
    }
    if (!E->cap_stream) CK(cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking));
    const int P = E->graph_period;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = CPH_OK;
    // the captured period starts at a step t with t % P == 1 (t > 0 throughout)
    for (int s = 0; s < P && rc == CPH_OK; ++s) rc = enqueue_step(E, 1 + s, s, true, E->cap_stream);
    if (rc == CPH_OK) rc = launch_tick(E, P, E->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(E->cap_stream, &g);
    if (rc != CPH_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return fail(E, CPH_E_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    cudaGraphExec_t ex = nullptr;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(E, CPH_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
    E->graph[mode] = ex;
    *out = ex;
    return CPH_OK;
}

} // namespace

namespace {

// Work items of the pair passes.  Ordered items: groups of kWarpAtoms atoms i
// (one warp each) of the walkers whose system runs the ordered passes.
// Symmetric items (FP32), for the other walkers: j-tile chunks of `chunk`
// tiles, every 256-atom i-tile against the 32-atom j-tiles from its first
// atom on.  Replaces the current item arrays and the device copy of the
// per-system shape flags, and drops captured graphs (they hold the old item
// pointers).
int build_items(cph_engine* E, int chunk) {
    // the pair passes sum i-side partials per aligned group of kSymG j-tiles:
    // items must start and end on group boundaries (or at the row's end)
    if (chunk < kSymG || chunk % kSymG != 0 || kSymI % (kSymG * kSymJ) != 0)
        return fail(E, CPH_E_INVALID, "work-item size %d is not a multiple of %d j-tiles", chunk, kSymG);
    const int W = E->V.W;
    std::vector<Item> oitems, o_by_w;
    std::vector<int> o_off(W + 1, 0);
    std::vector<int> ordered(E->n_sys);
    for (int s = 0; s < E->n_sys; ++s) ordered[s] = sys_ordered(E, s) ? 1 : 0;
    // FP64 arithmetic on few atoms (a small walker or two): four warps per atom,
    // one atom per CTA, so that the scarce FP64 units of every SM share the
    // work.  Counted over the whole grid, local or not, so that every engine of
    // a sharded grid sums in the same order.  (FP32 small systems measured no
    // faster this way: the staging of the j atoms, not the arithmetic, grows.)
    long long n_oatoms = 0;
    for (int w = 0; w < W; ++w)
        if (ordered[E->h_w_sys[w]]) n_oatoms += E->h_sys_n[E->h_w_sys[w]];
    E->ordered_wpa = (E->precision == CPH_PREC_FP64 && n_oatoms <= kOrderedFewAtoms) ? 4 : 1;
    const int apc = kWarpAtoms / E->ordered_wpa; // atoms per CTA
    for (int w = 0; w < W; ++w) {
        const int s = E->h_w_sys[w], N = E->h_sys_n[s];
        // the masked j-tiles of a group are those of the 128-atom i-tile it lies in
        if (ordered[s] && E->h_w_local[w])
            for (int i0 = 0; i0 < N; i0 += apc)
                o_by_w.push_back(Item{w, i0, E->h_sys_st_off[s] + i0 / kTile, 0});
        o_off[w + 1] = (int)o_by_w.size();
    }
    oitems = o_by_w;
    std::stable_sort(oitems.begin(), oitems.end(), [&](const Item& a, const Item& b) {
        return E->h_sys_n[E->h_w_sys[a.w]] > E->h_sys_n[E->h_w_sys[b.w]];
    });
    std::vector<SymItem> sym, by_w;
    std::vector<int> w_off(W + 1, 0);
    for (int w = 0; w < W; ++w) {
        const int s = E->h_w_sys[w], N = E->h_sys_n[s];
        if (ordered[s] || !E->h_w_local[w]) {
            w_off[w + 1] = (int)by_w.size();
            continue;
        }
        const int njt = (N + kSymJ - 1) / kSymJ;
        for (int it = 0; it * kSymI < N; ++it) {
            const int i0 = it * kSymI;
            for (int jt = i0 / kSymJ; jt < njt; jt += chunk)
                by_w.push_back(SymItem{w, i0, jt, std::min(njt, jt + chunk), E->h_sys_sst_off[s] + it, 0});
        }
        w_off[w + 1] = (int)by_w.size();
    }
    sym = by_w;
    std::stable_sort(sym.begin(), sym.end(), [](const SymItem& a, const SymItem& b) {
        return (a.jt1 - a.jt0) > (b.jt1 - b.jt0);
    });
    for (auto& g : E->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (E->d_sym) cudaFree(E->d_sym);
    if (E->d_sym_by_w) cudaFree(E->d_sym_by_w);
    E->d_sym = E->d_sym_by_w = nullptr;
    CK(cudaMalloc(&E->d_sym, sizeof(SymItem) * std::max<size_t>(1, sym.size())));
    CK(cudaMalloc(&E->d_sym_by_w, sizeof(SymItem) * std::max<size_t>(1, by_w.size())));
    CK(cudaMemcpy(E->d_sym, sym.data(), sizeof(SymItem) * sym.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(E->d_sym_by_w, by_w.data(), sizeof(SymItem) * by_w.size(), cudaMemcpyHostToDevice));
    E->n_sym = (int)sym.size();
    E->sym_w_off = w_off;
    E->sym_chunk = chunk;
    if (E->d_items) cudaFree(E->d_items);
    if (E->d_items_by_w) cudaFree(E->d_items_by_w);
    E->d_items = E->d_items_by_w = nullptr;
    CK(cudaMalloc(&E->d_items, sizeof(Item) * std::max<size_t>(1, oitems.size())));
    CK(cudaMalloc(&E->d_items_by_w, sizeof(Item) * std::max<size_t>(1, o_by_w.size())));
    CK(cudaMemcpy(E->d_items, oitems.data(), sizeof(Item) * oitems.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(E->d_items_by_w, o_by_w.data(), sizeof(Item) * o_by_w.size(), cudaMemcpyHostToDevice));
    E->n_items = (int)oitems.size();
    E->item_w_off = o_off;
    CK(cudaMemcpy(E->d_sys_ordered, ordered.data(), sizeof(int) * ordered.size(), cudaMemcpyHostToDevice));
    return CPH_OK;
}

} // namespace

// =====================================================================
// C ABI
// =====================================================================
extern "C" {

const char* cph_last_error(const cph_engine* e) { return e ? e->err.c_str() : g_last_error.c_str(); }

int cph_init_system(const cph_system_desc* sys, int n_sys, const cph_grid_desc* grid,
                    const cph_run_params* p, uint64_t seed, cph_engine** out) {
    if (!out) return fail(nullptr, CPH_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!sys || n_sys < 1 || !grid || !p) return fail(nullptr, CPH_E_INVALID, "missing descriptor");
    if (p->precision != CPH_PREC_FP32 && p->precision != CPH_PREC_FP64)
        return fail(nullptr, CPH_E_INVALID, "unknown precision %d", p->precision);
    if (!std::isfinite(p->gb.sa_gamma) || !(p->gb.sa_probe >= 0) || !std::isfinite(p->gb.sa_probe))
        return fail(nullptr, CPH_E_INVALID, "surface term: sa_gamma must be finite, sa_probe finite and >= 0");
    if (!(p->gb.kappa >= 0) || !std::isfinite(p->gb.kappa))
        return fail(nullptr, CPH_E_INVALID, "salt screening kappa must be finite and >= 0");
    if (!(p->gb.rgbmax >= 0) || !std::isfinite(p->gb.rgbmax))
        return fail(nullptr, CPH_E_INVALID, "Born-radius cutoff rgbmax must be finite and >= 0 (0 = none)");
    if (!(p->dt > 0) || !(p->gamma_ln >= 0) || !(p->gb.eps_in > 0) || !(p->gb.eps_out > 0))
        return fail(nullptr, CPH_E_INVALID, "dt, gamma_ln, eps_in, eps_out must be positive");
    if (p->mc_ph_every < 0 || p->mc_redox_every < 0 || p->exchange_every < 0)
        return fail(nullptr, CPH_E_INVALID, "negative interval");
    if (p->t_exchange_energy != CPH_TEX_POTENTIAL && p->t_exchange_energy != CPH_TEX_SEMIGRAND)
        return fail(nullptr, CPH_E_INVALID, "unknown T-exchange energy %d", p->t_exchange_energy);
    if (grid->nE < 1 || grid->npH < 1 || grid->nT < 1 || !grid->E || !grid->pH || !grid->T ||
        !grid->system_of_slot)
        return fail(nullptr, CPH_E_INVALID, "bad grid");
    if (grid->n_order < 1 || grid->n_order > 3) return fail(nullptr, CPH_E_INVALID, "n_order must be 1..3");
    for (int k = 0; k < grid->n_order; ++k)
        if (grid->order[k] < 0 || grid->order[k] > 2) return fail(nullptr, CPH_E_INVALID, "bad order entry");
    for (int k = 0; k < grid->nT; ++k)
        if (!(grid->T[k] > 0)) return fail(nullptr, CPH_E_INVALID, "temperatures must be positive");
    const int W = grid->nE * grid->npH * grid->nT;
    for (int w = 0; w < W; ++w)
        if (grid->system_of_slot[w] < 0 || grid->system_of_slot[w] >= n_sys)
            return fail(nullptr, CPH_E_INVALID, "system_of_slot[%d] out of range", w);

    // ---- validate systems and build per-system host tables
    std::vector<int> sys_n(n_sys), sys_poff(n_sys + 1, 0), sys_site_off(n_sys + 1, 0);
    std::vector<double> rho, rt, sc, sigh, sqe, mass, x0;
    std::vector<int> excl_off(1, 0), excl_j, bond_off(1, 0), bond_idx, bond_ij, ang_off(1, 0),
        ang_idx, ang_ijk;
    std::vector<double> bond_k, bond_r0, ang_k, ang_t0;
    // SHAKE clusters (system-local atom indices), concatenated over systems
    std::vector<int> shk_heavy, shk_off{0}, shk_h, shk_sys_off{0};
    std::vector<double> shk_d;
    if (p->shake && !(p->shake_tol > 0) )
        return fail(nullptr, CPH_E_INVALID, "shake_tol must be > 0 when shake is on");
    std::vector<int> site_kind, site_nat, site_aoff, site_atoms, site_nst, site_qoff, site_noff,
        site_np, site_ne, site_sys, site_init;
    std::vector<double> site_q, site_ref;
    std::vector<int> mt_off(1, 0), mt_list, sys_st_off(n_sys + 1, 0);
    std::vector<int> smt_off(1, 0), smt_list, sys_sst_off(n_sys + 1, 0);
    std::vector<int> sys_bond_off(n_sys + 1, 0), sys_ang_off(n_sys + 1, 0);
    const double off = p->gb.offset;
    for (int s = 0; s < n_sys; ++s) {
        const cph_system_desc& d = sys[s];
        const int N = d.n_atoms;
        if (N < 1 || N > 65536) return fail(nullptr, CPH_E_INVALID, "system %d: n_atoms %d out of 1..65536", s, N);
        if (!d.x || !d.mass || !d.q || !d.rho || !d.screen || !d.sigma || !d.eps)
            return fail(nullptr, CPH_E_INVALID, "system %d: missing per-atom array", s);
        if (!finite_all(d.x, 3 * (size_t)N) || !finite_all(d.q, N) || (d.v && !finite_all(d.v, 3 * (size_t)N)))
            return fail(nullptr, CPH_E_INVALID, "system %d: non-finite positions, velocities or charges", s);
        sys_n[s] = N;
        sys_poff[s + 1] = sys_poff[s] + N;
        for (int a = 0; a < N; ++a) {
            if (!(d.mass[a] > 0)) return fail(nullptr, CPH_E_INVALID, "system %d atom %d: mass must be > 0", s, a);
            if (!(d.rho[a] > off)) return fail(nullptr, CPH_E_INVALID, "system %d atom %d: rho must exceed the offset", s, a);
            if (!(d.screen[a] >= 0) || !(d.sigma[a] >= 0) || !(d.eps[a] >= 0))
                return fail(nullptr, CPH_E_INVALID, "system %d atom %d: negative screen, sigma or eps", s, a);
            rho.push_back(d.rho[a]);
            rt.push_back(d.rho[a] - off);
            sc.push_back(d.screen[a] * (d.rho[a] - off));
            sigh.push_back(0.5 * d.sigma[a]);
            sqe.push_back(std::sqrt(d.eps[a]));
            mass.push_back(d.mass[a]);
            for (int c = 0; c < 3; ++c) x0.push_back(d.x[3 * a + c]);
        }
        // exclusions: 1-2 and 1-3 through the bond graph, plus the extra list
        std::vector<std::vector<int>> nb(N);
        if (d.n_bonds < 0 || (d.n_bonds > 0 && (!d.bonds || !d.bond_k || !d.bond_r0)))
            return fail(nullptr, CPH_E_INVALID, "system %d: bad bond arrays", s);
        const int bond_base = (int)bond_k.size();
        std::vector<std::vector<std::pair<int, double>>> hyd(N); // SHAKE: hydrogens per heavy atom
        for (int b = 0; b < d.n_bonds; ++b) {
            int i = d.bonds[2 * b], j = d.bonds[2 * b + 1];
            if (i < 0 || j < 0 || i >= N || j >= N || i == j)
                return fail(nullptr, CPH_E_INVALID, "system %d: bond %d has bad atoms", s, b);
            nb[i].push_back(j);
            nb[j].push_back(i);
            bond_ij.push_back(i);
            bond_ij.push_back(j);
            const bool hi = d.mass[i] < 2.0, hj = d.mass[j] < 2.0;
            const bool con = p->shake && (hi || hj);
            if (con) {
                if (hi && hj)
                    return fail(nullptr, CPH_E_INVALID, "system %d: bond %d joins two hydrogens (cannot be constrained)", s, b);
                if (!(d.bond_r0[b] > 0))
                    return fail(nullptr, CPH_E_INVALID, "system %d: constrained bond %d needs r0 > 0", s, b);
                hyd[hi ? j : i].push_back({hi ? i : j, d.bond_r0[b]});
            }
            bond_k.push_back(con ? 0.0 : d.bond_k[b]); // constrained: no harmonic term
            bond_r0.push_back(d.bond_r0[b]);
        }
        // clusters must not share atoms (one thread owns each): a hydrogen may be
        // constrained to one heavy atom only
        std::vector<char> owned(N, 0);
        for (int a = 0; a < N; ++a) {
            if (hyd[a].empty()) continue;
            if (hyd[a].size() > 8)
                return fail(nullptr, CPH_E_INVALID, "system %d: atom %d carries more than 8 constrained hydrogens", s, a);
            shk_heavy.push_back(a);
            for (auto& hd : hyd[a]) {
                if (owned[hd.first]++)
                    return fail(nullptr, CPH_E_INVALID, "system %d: hydrogen %d is bonded to two heavy atoms", s, hd.first);
                shk_h.push_back(hd.first);
                shk_d.push_back(hd.second);
            }
            shk_off.push_back((int)shk_h.size());
        }
        shk_sys_off.push_back((int)shk_heavy.size());
        std::vector<std::set<int>> ex(N);
        for (int i = 0; i < N; ++i)
            for (int j : nb[i]) {
                ex[i].insert(j);
                for (int k : nb[j])
                    if (k != i) ex[i].insert(k);
            }
        if (d.n_excl < 0 || (d.n_excl > 0 && !d.excl)) return fail(nullptr, CPH_E_INVALID, "system %d: bad exclusion list", s);
        for (int e = 0; e < d.n_excl; ++e) {
            int i = d.excl[2 * e], j = d.excl[2 * e + 1];
            if (i < 0 || j < 0 || i >= N || j >= N || i == j)
                return fail(nullptr, CPH_E_INVALID, "system %d: exclusion %d has bad atoms", s, e);
            ex[i].insert(j);
            ex[j].insert(i);
        }
        for (int i = 0; i < N; ++i) {
            for (int j : ex[i]) excl_j.push_back(j);
            excl_off.push_back((int)excl_j.size());
        }
        // bonded term lists per atom
        std::vector<std::vector<int>> bt(N), at(N);
        for (int b = 0; b < d.n_bonds; ++b) {
            bt[d.bonds[2 * b]].push_back(bond_base + b);
            bt[d.bonds[2 * b + 1]].push_back(bond_base + b);
        }
        if (d.n_angles < 0 || (d.n_angles > 0 && (!d.angles || !d.angle_k || !d.angle_t0)))
            return fail(nullptr, CPH_E_INVALID, "system %d: bad angle arrays", s);
        const int ang_base = (int)ang_k.size();
        for (int a = 0; a < d.n_angles; ++a) {
            int i = d.angles[3 * a], j = d.angles[3 * a + 1], k = d.angles[3 * a + 2];
            if (i < 0 || j < 0 || k < 0 || i >= N || j >= N || k >= N || i == j || j == k || i == k)
                return fail(nullptr, CPH_E_INVALID, "system %d: angle %d has bad atoms", s, a);
            ang_ijk.push_back(i);
            ang_ijk.push_back(j);
            ang_ijk.push_back(k);
            ang_k.push_back(d.angle_k[a]);
            ang_t0.push_back(d.angle_t0[a]);
            at[i].push_back(ang_base + a);
            at[j].push_back(ang_base + a);
            at[k].push_back(ang_base + a);
        }
        sys_bond_off[s + 1] = (int)bond_k.size();
        sys_ang_off[s + 1] = (int)ang_k.size();
        for (int i = 0; i < N; ++i) {
            for (int b : bt[i]) bond_idx.push_back(b);
            bond_off.push_back((int)bond_idx.size());
            for (int a : at[i]) ang_idx.push_back(a);
            ang_off.push_back((int)ang_idx.size());
        }
        // masked j-tiles per i-tile: self and excluded partners
        const int nt = (N + kTile - 1) / kTile;
        sys_st_off[s + 1] = sys_st_off[s] + nt;
        for (int it = 0; it < nt; ++it) {
            std::set<int> tiles;
            for (int i = it * kTile; i < std::min(N, (it + 1) * kTile); ++i) {
                tiles.insert(i / kTile);
                for (int j : ex[i]) tiles.insert(j / kTile);
            }
            for (int jt : tiles) mt_list.push_back(jt);
            mt_off.push_back((int)mt_list.size());
        }
        // symmetric passes: masked 32-atom j-tiles per 256-atom i-tile (diagonal
        // block, partners beyond j > i that are excluded)
        const int nts = (N + kSymI - 1) / kSymI;
        sys_sst_off[s + 1] = sys_sst_off[s] + nts;
        for (int it = 0; it < nts; ++it) {
            std::set<int> tiles;
            const int i0 = it * kSymI, i1 = std::min(N, i0 + kSymI);
            for (int jt = i0 / kSymJ; jt * kSymJ < i1; ++jt) tiles.insert(jt);
            for (int i = i0; i < i1; ++i)
                for (int j : ex[i])
                    if (j > i) tiles.insert(j / kSymJ);
            for (int jt : tiles) smt_list.push_back(jt);
            smt_off.push_back((int)smt_list.size());
        }
        // sites
        if (d.n_sites < 0 || (d.n_sites > 0 && !d.sites)) return fail(nullptr, CPH_E_INVALID, "system %d: bad site list", s);
        std::vector<char> used(N, 0);
        for (int k = 0; k < d.n_sites; ++k) {
            const cph_site_desc& sd = d.sites[k];
            if (sd.kind != CPH_SITE_PH && sd.kind != CPH_SITE_REDOX)
                return fail(nullptr, CPH_E_INVALID, "system %d site %d: bad kind", s, k);
            if (sd.n_atoms < 1 || sd.n_atoms > kMaxSiteAtoms || !sd.atoms || !sd.q || !sd.n_prot || !sd.n_elec)
                return fail(nullptr, CPH_E_INVALID, "system %d site %d: n_atoms must be 1..%d with all arrays", s, k, kMaxSiteAtoms);
            if (sd.n_states < 2 || sd.n_states > 8 || sd.init_state < 0 || sd.init_state >= sd.n_states)
                return fail(nullptr, CPH_E_INVALID, "system %d site %d: n_states must be 2..8 and init_state valid", s, k);
            if (!finite_all(sd.q, (size_t)sd.n_states * sd.n_atoms) || !std::isfinite(sd.ref))
                return fail(nullptr, CPH_E_INVALID, "system %d site %d: non-finite charges or reference", s, k);
            site_kind.push_back(sd.kind);
            site_nat.push_back(sd.n_atoms);
            site_aoff.push_back((int)site_atoms.size());
            site_nst.push_back(sd.n_states);
            site_qoff.push_back((int)site_q.size());
            site_noff.push_back((int)site_np.size());
            site_ref.push_back(sd.ref);
            site_sys.push_back(s);
            site_init.push_back(sd.init_state);
            for (int m = 0; m < sd.n_atoms; ++m) {
                int a = sd.atoms[m];
                if (a < 0 || a >= N || used[a])
                    return fail(nullptr, CPH_E_INVALID, "system %d site %d: atom %d invalid or shared", s, k, a);
                used[a] = 1;
                site_atoms.push_back(a);
            }
            for (int q = 0; q < sd.n_states * sd.n_atoms; ++q) site_q.push_back(sd.q[q]);
            for (int st = 0; st < sd.n_states; ++st) {
                site_np.push_back(sd.n_prot[st]);
                site_ne.push_back(sd.n_elec[st]);
            }
        }
        sys_site_off[s + 1] = sys_site_off[s] + d.n_sites;
    }

    // ---- walkers
    std::vector<int> w_sys(W), w_off(W + 1, 0), w_site_off(W + 1, 0), a_walker;
    for (int w = 0; w < W; ++w) {
        w_sys[w] = grid->system_of_slot[w];
        w_off[w + 1] = w_off[w] + sys_n[w_sys[w]];
        w_site_off[w + 1] = w_site_off[w] + (sys_site_off[w_sys[w] + 1] - sys_site_off[w_sys[w]]);
    }
    const long long total_ll = w_off[W];
    if (total_ll > (1ll << 30)) return fail(nullptr, CPH_E_INVALID, "too many atoms in total");
    const int total = (int)total_ll;
    a_walker.resize(total);
    std::vector<double> hx(3 * (size_t)total), hv(3 * (size_t)total, 0.0), hq(total);
    std::vector<int> hstate(w_site_off[W]);
    for (int w = 0; w < W; ++w) {
        const cph_system_desc& d = sys[w_sys[w]];
        for (int a = 0; a < d.n_atoms; ++a) {
            a_walker[w_off[w] + a] = w;
            hq[w_off[w] + a] = d.q[a];
            for (int c = 0; c < 3; ++c) {
                hx[3 * (size_t)(w_off[w] + a) + c] = d.x[3 * a + c];
                if (d.v) hv[3 * (size_t)(w_off[w] + a) + c] = d.v[3 * a + c];
            }
        }
        for (int k = 0; k < d.n_sites; ++k) {
            const cph_site_desc& sd = d.sites[k];
            hstate[w_site_off[w] + k] = sd.init_state;
            for (int m = 0; m < sd.n_atoms; ++m) hq[w_off[w] + sd.atoms[m]] = sd.q[sd.init_state * sd.n_atoms + m];
        }
    }
    cph_engine* E = new cph_engine();
    std::unique_ptr<cph_engine> guard(E);
    E->precision = p->precision;
    E->mc_ph = p->mc_ph_every;
    E->mc_redox = p->mc_redox_every;
    E->ex_every = p->exchange_every;
    E->n_sys = n_sys;
    E->h_sys_n = sys_n;
    E->h_w_sys = w_sys;
    E->h_w_off = w_off;
    E->h_w_site_off = w_site_off;
    E->h_sys_site_off = sys_site_off;
    E->h_site_nst = site_nst;
    E->h_site_kind = site_kind;
    E->h_site_noff = site_noff;
    E->h_site_np = site_np;
    E->h_site_ne = site_ne;
    E->n_site_states = (int)site_np.size();
    E->h_sys_sst_off = sys_sst_off;
    E->h_sys_st_off = sys_st_off;
    E->h_sys_shape.assign(n_sys, CPH_SHAPE_SYMMETRIC);
    E->graph_period = schedule_period(E);
    View& V = E->V;
    V.W = W;
    V.total_atoms = total;
    std::vector<int> sys_poff_v(sys_poff.begin(), sys_poff.end());
    int* d;
    double* dd;
    TRY(upload(E, w_sys, &d)); V.w_sys = d;
    TRY(upload(E, w_off, &d)); V.w_off = d;
    TRY(upload(E, a_walker, &d)); V.a_walker = d;
    TRY(upload(E, w_site_off, &d)); V.w_site_off = d;
    TRY(upload(E, sys_n, &d)); V.sys_n = d;
    TRY(upload(E, sys_poff_v, &d)); V.sys_poff = d;
    TRY(upload(E, sys_site_off, &d)); V.sys_site_off = d;
    TRY(upload(E, rho, &dd)); V.rho = dd;
    TRY(upload(E, rt, &dd)); V.rt = dd;
    {
        std::vector<double> irt(rt.size()), irho(rho.size());
        for (size_t q = 0; q < rt.size(); ++q) irt[q] = 1.0 / rt[q];
        for (size_t q = 0; q < rho.size(); ++q) irho[q] = 1.0 / rho[q];
        TRY(upload(E, irt, &dd)); V.irt = dd;
        TRY(upload(E, irho, &dd)); V.irho = dd;
    }
    TRY(upload(E, sc, &dd)); V.sc = dd;
    TRY(upload(E, sigh, &dd)); V.sigh = dd;
    TRY(upload(E, sqe, &dd)); V.sqe = dd;
    TRY(upload(E, mass, &dd)); V.mass = dd;
    {
        std::vector<float4> pb(rt.size());
        std::vector<float2> pl(rt.size());
        for (size_t p = 0; p < rt.size(); ++p) {
            pb[p] = make_float4((float)sc[p], (float)rt[p], (float)(1.0 / rt[p]), 0.f);
            pl[p] = make_float2((float)sigh[p], (float)sqe[p]);
        }
        float4* d4;
        float2* d2;
        TRY(upload(E, pb, &d4)); V.pb32 = d4;
        TRY(upload(E, pl, &d2)); V.plj32 = d2;
    }
    TRY(upload(E, excl_off, &d)); V.excl_off = d;
    TRY(upload(E, excl_j, &d)); V.excl_j = d;
    TRY(upload(E, bond_off, &d)); V.bond_off = d;
    TRY(upload(E, bond_idx, &d)); V.bond_idx = d;
    TRY(upload(E, bond_ij, &d)); V.bond_ij = d;
    TRY(upload(E, bond_k, &dd)); V.bond_k = dd;
    TRY(upload(E, bond_r0, &dd)); V.bond_r0 = dd;
    TRY(upload(E, ang_off, &d)); V.ang_off = d;
    TRY(upload(E, ang_idx, &d)); V.ang_idx = d;
    TRY(upload(E, ang_ijk, &d)); V.ang_ijk = d;
    TRY(upload(E, ang_k, &dd)); V.ang_k = dd;
    TRY(upload(E, ang_t0, &dd)); V.ang_t0 = dd;
    {
        std::vector<double2> cs0(ang_t0.size());
        for (size_t a = 0; a < ang_t0.size(); ++a) cs0[a] = make_double2(std::cos(ang_t0[a]), std::sin(ang_t0[a]));
        double2* dcs;
        TRY(upload(E, cs0, &dcs)); V.ang_cs0 = dcs;
    }
    TRY(upload(E, sys_bond_off, &d)); V.sys_bond_off = d;
    TRY(upload(E, sys_ang_off, &d)); V.sys_ang_off = d;
    {
        std::vector<long long> tf_off(W + 1, 0);
        for (int w = 0; w < W; ++w) {
            const int s = w_sys[w];
            const int nb = sys_bond_off[s + 1] - sys_bond_off[s], na = sys_ang_off[s + 1] - sys_ang_off[s];
            tf_off[w + 1] = tf_off[w] + 6LL * nb + 9LL * na;
            E->max_terms = std::max(E->max_terms, nb + na);
        }
        long long* dtf;
        TRY(upload(E, tf_off, &dtf)); V.w_tf_off = dtf;
        float* dtfb;
        TRY(alloc0(E, (size_t)tf_off[W], &dtfb)); V.tforce = dtfb;
    }
    TRY(upload(E, mt_off, &d)); V.mt_off = d;
    TRY(upload(E, mt_list, &d)); V.mt_list = d;
    TRY(upload(E, smt_off, &d)); V.smt_off = d;
    TRY(upload(E, smt_list, &d)); V.smt_list = d;
    TRY(upload(E, site_kind, &d)); V.site_kind = d;
    TRY(upload(E, site_nat, &d)); V.site_nat = d;
    TRY(upload(E, site_aoff, &d)); V.site_aoff = d;
    TRY(upload(E, site_atoms, &d)); V.site_atoms = d;
    TRY(upload(E, site_nst, &d)); V.site_nst = d;
    TRY(upload(E, site_qoff, &d)); V.site_qoff = d;
    TRY(upload(E, site_noff, &d)); V.site_noff = d;
    TRY(upload(E, site_q, &dd)); V.site_q = dd;
    TRY(upload(E, site_np, &d)); V.site_np = d;
    TRY(upload(E, site_ne, &d)); V.site_ne = d;
    TRY(upload(E, site_ref, &dd)); V.site_ref = dd;
    TRY(alloc0(E, site_np.size(), &dd)); V.site_uref = dd;
    TRY(upload(E, hx, &dd)); V.x = dd;
    TRY(upload(E, hv, &dd)); V.v = dd;
    TRY(upload(E, hq, &dd)); V.q = dd;
    TRY(alloc0(E, total, &dd)); V.psi = dd;
    TRY(alloc0(E, total, &dd)); V.R = dd;
    TRY(alloc0(E, total, &dd)); V.dRdpsi = dd;
    TRY(alloc0(E, total, &dd)); V.c = dd;
    TRY(alloc0(E, 3 * (size_t)total, &dd)); V.Fd = dd;
    TRY(alloc0(E, 3 * (size_t)total, &dd)); V.F = dd;
    long long* dfx;
    TRY(alloc0(E, 3 * (size_t)total, &dfx)); V.Ffix = dfx;
    TRY(alloc0(E, (size_t)total, &dfx)); V.dRfix = dfx;
    TRY(alloc0(E, (size_t)total, &dfx)); V.Hfix = dfx;
    {
        float4* d4;
        float* d1;
        TRY(alloc0(E, (size_t)total, &d4)); V.xs = d4;
        TRY(alloc0(E, (size_t)total, &d4)); V.gq = d4;
        TRY(alloc0(E, (size_t)total, &d1)); V.c32 = d1;
    }
    long long* dl;
    TRY(alloc0(E, (size_t)W * kEAcc, &dl)); V.eacc = dl;
    std::vector<int> ident(W);
    std::iota(ident.begin(), ident.end(), 0);
    TRY(upload(E, ident, &d)); V.slot_of = d;
    TRY(upload(E, ident, &d)); V.walker_at = d;
    TRY(upload(E, hstate, &d)); V.site_state = d;
    std::vector<double> ones(W, 1.0);
    TRY(upload(E, ones, &dd)); V.vscale = dd;
    TRY(alloc0(E, 1, &dl)); V.step = dl;
    TRY(alloc0(E, 1, &d)); V.status = d;
    TRY(alloc0(E, 4, &d)); V.ex_state = d;
    TRY(alloc0(E, 10, &dl)); V.stats = dl;
    cph_mc_record* dm;
    {
        void* pm = nullptr;
        CK(cudaMalloc(&pm, std::max<size_t>(1, w_site_off[W]) * sizeof(cph_mc_record)));
        E->mem.ptrs.push_back(pm);
        CK(cudaMemset(pm, 0xff, std::max<size_t>(1, w_site_off[W]) * sizeof(cph_mc_record)));
        dm = (cph_mc_record*)pm;
    }
    V.mc_rec = dm;
    {
        // per (walker, site) scratch of the two-kernel MC sweep
        const size_t nsw = (size_t)w_site_off[W];
        int* di2;
        double* dd2;
        TRY(alloc0(E, nsw, &di2)); V.mc_from = di2;
        TRY(alloc0(E, nsw, &di2)); V.mc_to = di2;
        TRY(alloc0(E, nsw, &di2)); V.mc_take = di2;
        TRY(alloc0(E, nsw, &dd2)); V.mc_lnu = dd2;
        TRY(alloc0(E, nsw, &dd2)); V.mc_du0 = dd2;
        for (int s = 0; s < n_sys; ++s) E->max_sites = std::max(E->max_sites, sys_site_off[s + 1] - sys_site_off[s]);
    }
    E->ex_cap = W; // pairs per attempt <= slots / 2
    {
        void* pe = nullptr;
        CK(cudaMalloc(&pe, std::max<size_t>(1, E->ex_cap) * sizeof(cph_exchange_record)));
        E->mem.ptrs.push_back(pe);
        V.ex_rec = (cph_exchange_record*)pe;
    }
    TRY(alloc0(E, 1, &d)); V.ex_n = d;
    TRY(alloc0(E, std::max<size_t>(1, (size_t)w_site_off[W] * CPH_MAX_STATES), &dl)); V.occ = dl;
    if (p->shake) {
        std::vector<int> iw, ic;
        E->h_shk_w_off.assign(1, 0);
        for (int w = 0; w < W; ++w) {
            const int sy = E->h_w_sys[w];
            for (int c = shk_sys_off[sy]; c < shk_sys_off[sy + 1]; ++c) {
                iw.push_back(w);
                ic.push_back(c);
            }
            E->h_shk_w_off.push_back((int)iw.size());
        }
        TRY(upload(E, shk_heavy, &d)); V.shk_heavy = d;
        TRY(upload(E, shk_off, &d)); V.shk_off = d;
        TRY(upload(E, shk_h, &d)); V.shk_h = d;
        TRY(upload(E, shk_d, &dd)); V.shk_d = dd;
        TRY(upload(E, iw, &d)); V.shk_item_w = d;
        TRY(upload(E, ic, &d)); V.shk_item_c = d;
        TRY(alloc0(E, 3 * (size_t)total, &dd)); V.xprev = dd;
        V.shake_tol = p->shake_tol;
        E->n_shk = (int)iw.size();
    }
    TRY(alloc0(E, (size_t)W * W, &dl)); V.visits = dl;
    TRY(alloc0(E, 1, &dl)); V.n_obs = dl;
    std::vector<double> gE(grid->E, grid->E + grid->nE), gpH(grid->pH, grid->pH + grid->npH),
        gT(grid->T, grid->T + grid->nT);
    TRY(upload(E, gE, &dd)); V.gE = dd;
    TRY(upload(E, gpH, &dd)); V.gpH = dd;
    TRY(upload(E, gT, &dd)); V.gT = dd;
    V.nE = grid->nE;
    V.npH = grid->npH;
    V.nT = grid->nT;
    V.n_order = grid->n_order;
    for (int k = 0; k < 3; ++k) V.order[k] = k < grid->n_order ? grid->order[k] : 0;
    V.tau = 1.0 / p->gb.eps_in - 1.0 / p->gb.eps_out;
    V.kappa = p->gb.kappa;
    V.inv_eps_out = 1.0 / p->gb.eps_out;
    V.tau_pair = p->gb.kappa > 0 ? 1.0 : V.tau;
    V.sa_gamma = p->gb.sa_gamma;
    V.sa_probe = p->gb.sa_probe;
    V.rgbmax = p->gb.rgbmax > 0 ? p->gb.rgbmax : INFINITY;
    V.inv_eps_in = 1.0 / p->gb.eps_in;
    V.tau32 = (float)V.tau;
    V.iei32 = (float)V.inv_eps_in;
    V.ieo32 = (float)V.inv_eps_out;
    V.kappa32 = (float)V.kappa;
    V.sqk32 = (float)std::sqrt(kCoulomb);
    V.sqrt_k = std::sqrt(kCoulomb);
    V.alpha = p->gb.alpha;
    V.beta = p->gb.beta;
    V.gamma = p->gb.gamma;
    V.offset = p->gb.offset;
    V.dt = p->dt;
    V.gamma_ln = p->gamma_ln;
    V.lg_c1 = 1.0 - 0.5 * p->gamma_ln * p->dt;
    V.lg_c2 = 1.0 / (1.0 + 0.5 * p->gamma_ln * p->dt);
    {
        std::vector<double> im(mass.size()), sf(mass.size()), sqT(grid->nT);
        for (size_t a = 0; a < mass.size(); ++a) {
            im[a] = p->dt * kAccel / mass[a];
            sf[a] = std::sqrt(2.0 * p->gamma_ln * kBoltzmann * kAccel * p->dt / mass[a]);
        }
        for (int k = 0; k < grid->nT; ++k) sqT[k] = std::sqrt(grid->T[k]);
        TRY(upload(E, im, &dd)); V.lg_im = dd;
        TRY(upload(E, sf, &dd)); V.lg_sf = dd;
        TRY(upload(E, sqT, &dd)); V.lg_sqT = dd;
    }
    {
        double smax = 0.0, rtmax = 0.0;
        for (double v : sc) smax = std::max(smax, v);
        for (double v : rt) rtmax = std::max(rtmax, v);
        const double rfar = std::max(smax / (double)kHctXmax, smax + rtmax) * (1.0 + 1e-5);
        V.rfar2 = (float)(rfar * rfar);
        V.smax32 = (float)smax;
    }
    V.seed = seed;
    V.tex_semigrand = p->t_exchange_energy == CPH_TEX_SEMIGRAND ? 1 : 0;
    {
        int* dso;
        TRY(alloc0(E, (size_t)n_sys, &dso));
        E->d_sys_ordered = dso;
        V.sys_ordered = dso;
        E->h_w_local.assign(W, 1);
        int* dwl;
        TRY(upload(E, E->h_w_local, &dwl));
        E->d_w_local = dwl;
        V.w_local = dwl;
        V.first_local = 0;
        cph_exchange_row* drw;
        TRY(alloc0(E, (size_t)W, &drw));
        E->d_rows = drw;
        V.ex_rows = drw;
    }
    TRY(build_items(E, kSymChunk));

    // reference energies of every (site, state)
    if (!site_np.empty()) {
        std::vector<int> js, jst;
        for (size_t g = 0; g < site_nst.size(); ++g)
            for (int st = 0; st < site_nst[g]; ++st) {
                js.push_back((int)g);
                jst.push_back(st);
            }
        double* dx0;
        int *djs, *djst, *dss;
        TRY(upload(E, x0, &dx0));
        TRY(upload(E, js, &djs));
        TRY(upload(E, jst, &djst));
        TRY(upload(E, site_sys, &dss));
        const int nj = (int)js.size();
        k_site_ref<<<(nj + 63) / 64, 64>>>(E->V, dx0, djs, djst, dss, nj);
        CK(cudaGetLastError());
    }
    CK(cudaDeviceSynchronize());
    *out = guard.release();
    return CPH_OK;
}

void cph_destroy(cph_engine* e) { delete e; }

int cph_num_walkers(const cph_engine* e) { return e ? e->V.W : CPH_E_INVALID; }
int cph_total_atoms(const cph_engine* e) { return e ? e->V.total_atoms : CPH_E_INVALID; }

int cph_walker_offsets(const cph_engine* e, int* offsets) {
    if (!e || !offsets) return fail(nullptr, CPH_E_INVALID, "NULL argument");
    std::copy(e->h_w_off.begin(), e->h_w_off.end(), offsets);
    return CPH_OK;
}

int cph_site_offsets(const cph_engine* e, int* offsets) {
    if (!e || !offsets) return fail(nullptr, CPH_E_INVALID, "NULL argument");
    std::copy(e->h_w_site_off.begin(), e->h_w_site_off.end(), offsets);
    return CPH_OK;
}

int cph_set_launch_mode(cph_engine* e, int mode) {
    if (!e || (mode != CPH_LAUNCH_BATCHED && mode != CPH_LAUNCH_PER_REPLICA))
        return fail(e, CPH_E_INVALID, "bad launch mode");
    e->launch_mode = mode;
    return CPH_OK;
}

int cph_set_replica_streams(cph_engine* e, int n) {
    if (!e || n < 1 || n > 32) return fail(e, CPH_E_INVALID, "replica streams must be 1..32");
    cph_engine* E = e;
    if (!e->ev_fork) CK(cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming));
    for (int k = 0; k < n; ++k) {
        if (!e->rs[k]) CK(cudaStreamCreateWithFlags(&e->rs[k], cudaStreamNonBlocking));
        if (!e->ev_join[k]) CK(cudaEventCreateWithFlags(&e->ev_join[k], cudaEventDisableTiming));
    }
    if (n != e->n_rs && e->graph[1]) { // the per-replica graph was captured on the old streams
        cudaGraphExecDestroy(e->graph[1]);
        e->graph[1] = nullptr;
    }
    e->n_rs = n;
    return CPH_OK;
}

int cph_evaluate(cph_engine* e, void* stream) {
    if (!e) return fail(nullptr, CPH_E_INVALID, "NULL engine");
    return launch_forces(e, true, (cudaStream_t)stream, false, 0, 0);
}

int cph_time_passes(cph_engine* e, int reps, double* ms, void* stream) {
    if (!e || !ms || reps < 1) return fail(e, CPH_E_INVALID, "bad arguments");
    cph_engine* E = e;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[4];
    for (auto& x : ev) CK(cudaEventCreate(&x));
    double acc[3] = {0, 0, 0};
    int rc = CPH_OK;
    for (int r = 0; r < reps && rc == CPH_OK; ++r) {
        for (int p = 0; p < 3 && rc == CPH_OK; ++p) {
            cudaEventRecord(ev[p], st);
            rc = launch_pass(e, p, false, st);
        }
        cudaEventRecord(ev[3], st);
        cudaError_t ce = cudaEventSynchronize(ev[3]);
        if (ce != cudaSuccess && rc == CPH_OK) rc = fail(e, CPH_E_CUDA, "timing: %s", cudaGetErrorString(ce));
        for (int k = 0; k < 3 && rc == CPH_OK; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    if (rc != CPH_OK) return rc;
    for (int k = 0; k < 3; ++k) ms[k] = acc[k] / reps;
    return CPH_OK;
}

int cph_autotune(cph_engine* e, void* stream, int* chosen) {
    if (!e) return fail(nullptr, CPH_E_INVALID, "NULL engine");
    if (e->precision != CPH_PREC_FP32) {
        if (chosen) *chosen = 0;
        return CPH_OK; // the FP64 passes have no tunable shape
    }
    cph_engine* E = e;
    auto timed = [&](double* t) -> int {
        double ms[3];
        TRY(cph_time_passes(e, 1, ms, stream)); // warm-up
        TRY(cph_time_passes(e, 2, ms, stream));
        *t = ms[0] + ms[1] + ms[2];
        return CPH_OK;
    };
    // 1. work-item size of the symmetric tiles, every system symmetric
    const std::vector<int> shapes0 = e->h_sys_shape;
    e->h_sys_shape.assign(e->n_sys, CPH_SHAPE_SYMMETRIC);
    const int cand[] = {8, 16, 24, 32, 48, 64, 96, 128};
    double best = 1e300;
    int best_c = e->sym_chunk;
    for (int c : cand) {
        TRY(build_items(e, c));
        double t;
        TRY(timed(&t));
        if (t < best) {
            best = t;
            best_c = c;
        }
    }
    // 2. systems of at most n atoms on one warp per atom, n over the sizes
    std::vector<int> sizes(e->h_sys_n.begin(), e->h_sys_n.end());
    std::sort(sizes.begin(), sizes.end());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    int best_n = 0;
    for (int n : sizes) {
        for (int s = 0; s < e->n_sys; ++s)
            e->h_sys_shape[s] = e->h_sys_n[s] <= n ? CPH_SHAPE_WARP_PER_ATOM : CPH_SHAPE_SYMMETRIC;
        TRY(build_items(e, best_c));
        double t;
        TRY(timed(&t));
        if (t < best) {
            best = t;
            best_n = n;
        }
    }
    for (int s = 0; s < e->n_sys; ++s)
        e->h_sys_shape[s] = e->h_sys_n[s] <= best_n ? CPH_SHAPE_WARP_PER_ATOM : CPH_SHAPE_SYMMETRIC;
    (void)shapes0;
    TRY(build_items(e, best_c));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (chosen) *chosen = best_c;
    return CPH_OK;
}

int cph_set_tile_shape(cph_engine* e, int system, int shape) {
    if (!e) return fail(nullptr, CPH_E_INVALID, "NULL engine");
    if (system < 0 || system >= e->n_sys) return fail(e, CPH_E_INVALID, "system %d out of range", system);
    if (shape != CPH_SHAPE_SYMMETRIC && shape != CPH_SHAPE_WARP_PER_ATOM)
        return fail(e, CPH_E_INVALID, "unknown tile shape %d", shape);
    if (e->h_sys_shape[system] == shape) return CPH_OK;
    e->h_sys_shape[system] = shape;
    return build_items(e, e->sym_chunk);
}

int cph_set_local_walkers(cph_engine* e, int n, const int* walkers) {
    if (!e || n < 1 || n > e->V.W || !walkers) return fail(e, CPH_E_INVALID, "bad arguments");
    cph_engine* E = e;
    std::vector<int> m(e->V.W, 0);
    for (int k = 0; k < n; ++k) {
        if (walkers[k] < 0 || walkers[k] >= e->V.W || m[walkers[k]])
            return fail(e, CPH_E_INVALID, "walker list: entry %d is out of range or repeated", k);
        m[walkers[k]] = 1;
    }
    e->h_w_local = m;
    e->sharded = n < e->V.W;
    int first = 0;
    while (!m[first]) ++first;
    e->V.first_local = first;
    CK(cudaMemcpy(e->d_w_local, m.data(), sizeof(int) * m.size(), cudaMemcpyHostToDevice));
    return build_items(e, e->sym_chunk);
}

int cph_exchange_rows(cph_engine* e, cph_exchange_row* rows, int max, int* n_out, void* stream) {
    if (!e || !rows || !n_out) return fail(e, CPH_E_INVALID, "bad arguments");
    cph_engine* E = e;
    int nl = 0;
    for (int w = 0; w < e->V.W; ++w) nl += e->h_w_local[w];
    if (max < nl) return fail(e, CPH_E_INVALID, "rows: room for %d, %d local walkers", max, nl);
    cudaStream_t st = (cudaStream_t)stream;
    TRY(launch_forces(e, true, st, false, 0, 0)); // energies at the current state
    TRY(launch_exchange_rows(e, st));
    std::vector<cph_exchange_row> all(e->V.W);
    CK(cudaMemcpyAsync(all.data(), e->d_rows, sizeof(cph_exchange_row) * all.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int k = 0;
    for (int w = 0; w < e->V.W; ++w)
        if (e->h_w_local[w]) rows[k++] = all[w];
    *n_out = nl;
    return CPH_OK;
}

int cph_exchange_apply(cph_engine* e, int dim, const cph_exchange_row* rows, int n_rows, void* stream) {
    if (!e || !rows || dim < -1 || dim > 2) return fail(e, CPH_E_INVALID, "bad arguments");
    cph_engine* E = e;
    const int W = e->V.W;
    if (n_rows != W) return fail(e, CPH_E_INVALID, "exchange rows: %d given, %d walkers", n_rows, W);
    std::vector<cph_exchange_row> all(W);
    std::vector<char> seen(W, 0);
    for (int k = 0; k < n_rows; ++k) {
        const int w = rows[k].walker;
        if (w < 0 || w >= W || seen[w]) return fail(e, CPH_E_INVALID, "exchange rows: walker %d missing or repeated", w);
        seen[w] = 1;
        all[w] = rows[k];
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(e->d_rows, all.data(), sizeof(cph_exchange_row) * W, cudaMemcpyHostToDevice, st));
    TRY(launch_exchange_only(e, dim, 0, st));
    const int n = e->V.total_atoms, bs = 256;
    k_vscale<<<(n + bs - 1) / bs, bs, 0, st>>>(e->V);
    k_vscale_reset<<<(W + bs - 1) / bs, bs, 0, st>>>(e->V);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st)); // the host rows may be reused once this returns
    return CPH_OK;
}

int cph_get_tile_shapes(const cph_engine* e, int* shapes) {
    if (!e || !shapes) return fail(nullptr, CPH_E_INVALID, "bad arguments");
    for (int s = 0; s < e->n_sys; ++s)
        shapes[s] = e->precision == CPH_PREC_FP64 ? CPH_SHAPE_WARP_PER_ATOM : e->h_sys_shape[s];
    return CPH_OK;
}

int cph_step_replicas(cph_engine* e, int64_t n_steps, void* stream) {
    if (!e || n_steps < 0) return fail(e, CPH_E_INVALID, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t s = 0; s < n_steps; ++s) TRY(enqueue_step(e, e->h_step + s, (int)s, false, st));
    if (n_steps) TRY(launch_tick(e, n_steps, st));
    e->h_step += n_steps;
    return CPH_OK;
}

int cph_mc_titrate(cph_engine* e, int kind, void* stream) {
    if (!e || kind < 1 || kind > 3) return fail(e, CPH_E_INVALID, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(launch_pass(e, 0, false, st));
    TRY(launch_mc(e, kind, 0, st));
    return CPH_OK;
}

int cph_attempt_exchanges(cph_engine* e, int dim, void* stream) {
    if (!e || dim < -1 || dim > 2) return fail(e, CPH_E_INVALID, "bad arguments");
    if (e->sharded)
        return fail(e, CPH_E_STATE, "sharded engine: exchanges go through cph_exchange_rows / cph_exchange_apply");
    cudaStream_t st = (cudaStream_t)stream;
    cph_engine* E = e;
    // energies at the current state (needed for T; cheap to keep uniform)
    TRY(launch_forces(e, true, st, false, 0, 0));
    TRY(launch_exchange(e, dim, 0, st));
    const int n = e->V.total_atoms, bs = 256;
    k_vscale<<<(n + bs - 1) / bs, bs, 0, st>>>(e->V);
    k_vscale_reset<<<(e->V.W + bs - 1) / bs, bs, 0, st>>>(e->V);
    CK(cudaGetLastError());
    return CPH_OK;
}

int cph_run(cph_engine* e, int64_t n_steps, void* stream) {
    if (!e || n_steps < 0) return fail(e, CPH_E_INVALID, "bad arguments");
    if (e->sharded && e->ex_every > 0) {
        const long long t0 = e->h_step, t1 = e->h_step + n_steps; // steps t0 .. t1 - 1
        long long first = (t0 <= 0 ? 1 : t0);
        first = (first + e->ex_every - 1) / e->ex_every * e->ex_every;
        if (first < t1)
            return fail(e, CPH_E_STATE, "sharded engine: step %lld is an exchange step; run it with "
                        "cph_exchange_rows / cph_exchange_apply / cph_step_replicas", first);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cph_engine* E = e;
    const int P = e->graph_period;
    int64_t done = 0;
    int64_t direct = 0; // steps launched directly since the last tick
    while (done < n_steps) {
        const long long t = e->h_step;
        if (P > 1 && t % P == 1 && n_steps - done >= P) {
            if (direct) {
                TRY(launch_tick(e, direct, st));
                direct = 0;
            }
            cudaGraphExec_t g;
            TRY(get_graph(e, &g));
            CK(cudaGraphLaunch(g, st));
            e->h_step += P;
            done += P;
            e->mc_kinds_last = (e->mc_ph > 0 ? CPH_MC_PH : 0) | (e->mc_redox > 0 ? CPH_MC_REDOX : 0);
        } else {
            TRY(enqueue_step(e, t, (int)direct, true, st));
            ++direct;
            ++e->h_step;
            ++done;
        }
    }
    if (direct) TRY(launch_tick(e, direct, st));
    return CPH_OK;
}

#define SYNC_OR_FAIL(e, stream)                                                                 \
    do {                                                                                        \
        cph_engine* E = (e);                                                                    \
        CK(cudaStreamSynchronize((cudaStream_t)(stream)));                                      \
    } while (0)

static int copy_out(cph_engine* e, void* dst, const void* src, size_t bytes, void* stream) {
    if (!e || !dst) return fail(e, CPH_E_INVALID, "NULL argument");
    cph_engine* E = e;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
    return CPH_OK;
}

static int copy_in(cph_engine* e, void* dst, const void* src, size_t bytes, void* stream) {
    if (!e || !src) return fail(e, CPH_E_INVALID, "NULL argument");
    cph_engine* E = e;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
    return CPH_OK;
}

int cph_get_energies(cph_engine* e, double* out, void* stream) {
    if (!e || !out) return fail(e, CPH_E_INVALID, "NULL argument");
    std::vector<long long> h((size_t)e->V.W * kEAcc);
    TRY(copy_out(e, h.data(), e->V.eacc, h.size() * sizeof(long long), stream));
    for (int w = 0; w < e->V.W; ++w) {
        long long tot = 0;
        for (int t = 0; t < kEAcc; ++t) {
            out[w * CPH_NTERMS + t] = (double)h[w * kEAcc + t] / kScaleE;
            tot += h[w * kEAcc + t];
        }
        out[w * CPH_NTERMS + CPH_E_TOTAL] = (double)tot / kScaleE;
    }
    return CPH_OK;
}

int cph_get_forces(cph_engine* e, double* out, void* stream) {
    return copy_out(e, out, e ? e->V.F : nullptr, 3 * sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_get_born_radii(cph_engine* e, double* out, void* stream) {
    return copy_out(e, out, e ? e->V.R : nullptr, sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_get_positions(cph_engine* e, double* out, void* stream) {
    return copy_out(e, out, e ? e->V.x : nullptr, 3 * sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_set_positions(cph_engine* e, const double* in, void* stream) {
    if (e && in && !finite_all(in, 3 * (size_t)e->V.total_atoms)) return fail(e, CPH_E_INVALID, "non-finite positions");
    return copy_in(e, e ? e->V.x : nullptr, in, 3 * sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_get_velocities(cph_engine* e, double* out, void* stream) {
    return copy_out(e, out, e ? e->V.v : nullptr, 3 * sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_set_velocities(cph_engine* e, const double* in, void* stream) {
    if (e && in && !finite_all(in, 3 * (size_t)e->V.total_atoms)) return fail(e, CPH_E_INVALID, "non-finite velocities");
    return copy_in(e, e ? e->V.v : nullptr, in, 3 * sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_get_charges(cph_engine* e, double* out, void* stream) {
    return copy_out(e, out, e ? e->V.q : nullptr, sizeof(double) * (e ? e->V.total_atoms : 0), stream);
}
int cph_get_site_states(cph_engine* e, int* out, void* stream) {
    return copy_out(e, out, e ? e->V.site_state : nullptr, sizeof(int) * (e ? e->h_w_site_off.back() : 0), stream);
}
int cph_set_site_states(cph_engine* e, const int* in, void* stream) {
    if (!e || !in) return fail(e, CPH_E_INVALID, "NULL argument");
    for (int w = 0; w < e->V.W; ++w) {
        const int s = e->h_w_sys[w];
        for (int g = e->h_sys_site_off[s], k = 0; g < e->h_sys_site_off[s + 1]; ++g, ++k) {
            int st = in[e->h_w_site_off[w] + k];
            if (st < 0 || st >= e->h_site_nst[g]) return fail(e, CPH_E_INVALID, "walker %d site %d: bad state %d", w, k, st);
        }
    }
    TRY(copy_in(e, e->V.site_state, in, sizeof(int) * e->h_w_site_off.back(), stream));
    cph_engine* E = e;
    k_charges_from_states<<<e->V.W, 64, 0, (cudaStream_t)stream>>>(e->V);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return CPH_OK;
}
int cph_get_counts(cph_engine* e, int* n_prot, int* n_elec, void* stream) {
    if (!e || !n_prot || !n_elec) return fail(e, CPH_E_INVALID, "NULL argument");
    cph_engine* E = e;
    int* tmp = nullptr;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    CK(cudaMalloc(&tmp, 2 * sizeof(int) * e->V.W));
    k_counts<<<(e->V.W + 127) / 128, 128, 0, (cudaStream_t)stream>>>(e->V, tmp, tmp + e->V.W);
    cudaError_t ce = cudaStreamSynchronize((cudaStream_t)stream);
    if (ce == cudaSuccess) ce = cudaMemcpy(n_prot, tmp, sizeof(int) * e->V.W, cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(n_elec, tmp + e->V.W, sizeof(int) * e->V.W, cudaMemcpyDeviceToHost);
    cudaFree(tmp);
    if (ce != cudaSuccess) return fail(e, CPH_E_CUDA, "counts: %s", cudaGetErrorString(ce));
    return CPH_OK;
}
int cph_get_condition_map(cph_engine* e, int* slot_of_walker, void* stream) {
    return copy_out(e, slot_of_walker, e ? e->V.slot_of : nullptr, sizeof(int) * (e ? e->V.W : 0), stream);
}
int cph_set_condition_map(cph_engine* e, const int* slot_of_walker, void* stream) {
    if (!e || !slot_of_walker) return fail(e, CPH_E_INVALID, "NULL argument");
    const int W = e->V.W;
    std::vector<int> inv(W, -1);
    for (int w = 0; w < W; ++w) {
        int s = slot_of_walker[w];
        if (s < 0 || s >= W || inv[s] >= 0) return fail(e, CPH_E_INVALID, "condition map is not a permutation");
        if (e->h_w_sys[w] != e->h_w_sys[s]) return fail(e, CPH_E_INVALID, "walker %d cannot sit at slot %d of another system", w, s);
        inv[s] = w;
    }
    TRY(copy_in(e, e->V.slot_of, slot_of_walker, sizeof(int) * W, stream));
    TRY(copy_in(e, e->V.walker_at, inv.data(), sizeof(int) * W, stream));
    return CPH_OK;
}
int cph_get_accept_stats(cph_engine* e, int64_t* out, void* stream) {
    return copy_out(e, out, e ? e->V.stats : nullptr, 10 * sizeof(long long), stream);
}
int cph_get_occupancy(cph_engine* e, int64_t* out, int64_t* n_samples, void* stream) {
    if (!e || !out) return fail(e, CPH_E_INVALID, "NULL argument");
    const size_t rows = (size_t)e->h_w_site_off.back();
    if (rows) TRY(copy_out(e, out, e->V.occ, rows * CPH_MAX_STATES * sizeof(long long), stream));
    if (n_samples) TRY(copy_out(e, n_samples, e->V.n_obs, sizeof(long long), stream));
    return CPH_OK;
}
int cph_get_visits(cph_engine* e, int64_t* out, void* stream) {
    if (!e || !out) return fail(e, CPH_E_INVALID, "NULL argument");
    return copy_out(e, out, e->V.visits, (size_t)e->V.W * e->V.W * sizeof(long long), stream);
}
int cph_get_fractions(cph_engine* e, double* out, void* stream) {
    if (!e || !out) return fail(e, CPH_E_INVALID, "NULL argument");
    const int W = e->V.W;
    const size_t rows = (size_t)e->h_w_site_off.back();
    std::vector<long long> occ(std::max<size_t>(1, rows * CPH_MAX_STATES));
    long long ns = 0;
    if (rows) TRY(copy_out(e, occ.data(), e->V.occ, rows * CPH_MAX_STATES * sizeof(long long), stream));
    TRY(copy_out(e, &ns, e->V.n_obs, sizeof(long long), stream));
    if (ns <= 0) return fail(e, CPH_E_STATE, "no observable sample taken yet");
    // rows of slot s follow the sites of the system that starts at slot s
    for (int s = 0; s < W; ++s) {
        const int sys = e->h_w_sys[s];
        for (int g = e->h_sys_site_off[sys], k = 0; g < e->h_sys_site_off[sys + 1]; ++g, ++k) {
            const int* n = (e->h_site_kind[g] == CPH_SITE_PH ? e->h_site_np.data() : e->h_site_ne.data()) +
                           e->h_site_noff[g];
            const int nst = e->h_site_nst[g];
            int lo = n[0], hi = n[0];
            for (int t = 1; t < nst; ++t) lo = std::min(lo, n[t]), hi = std::max(hi, n[t]);
            const size_t row = (size_t)e->h_w_site_off[s] + k;
            double acc = 0.0;
            if (hi > lo)
                for (int t = 0; t < nst; ++t)
                    acc += (double)occ[row * CPH_MAX_STATES + t] * (double)(n[t] - lo) / (double)(hi - lo);
            out[row] = acc / (double)ns;
        }
    }
    return CPH_OK;
}
int cph_reset_observables(cph_engine* e, void* stream) {
    if (!e) return fail(e, CPH_E_INVALID, "NULL argument");
    cph_engine* E = e;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rows = (size_t)e->h_w_site_off.back();
    if (rows) CK(cudaMemsetAsync(e->V.occ, 0, rows * CPH_MAX_STATES * sizeof(long long), st));
    CK(cudaMemsetAsync(e->V.visits, 0, (size_t)e->V.W * e->V.W * sizeof(long long), st));
    CK(cudaMemsetAsync(e->V.n_obs, 0, sizeof(long long), st));
    return CPH_OK;
}
int cph_get_reference_energies(cph_engine* e, double* out) {
    return copy_out(e, out, e ? e->V.site_uref : nullptr, sizeof(double) * (e ? e->n_site_states : 0), nullptr);
}
int cph_get_mc_records(cph_engine* e, cph_mc_record* out, int max, int* n_out, void* stream) {
    if (!e || !out || !n_out) return fail(e, CPH_E_INVALID, "NULL argument");
    const int n = std::min(max, e->h_w_site_off.back());
    *n_out = n;
    return copy_out(e, out, e->V.mc_rec, sizeof(cph_mc_record) * n, stream);
}
int cph_get_exchange_records(cph_engine* e, cph_exchange_record* out, int max, int* n_out, void* stream) {
    if (!e || !out || !n_out) return fail(e, CPH_E_INVALID, "NULL argument");
    int n = 0;
    TRY(copy_out(e, &n, e->V.ex_n, sizeof(int), stream));
    n = std::min(n, std::min(max, e->ex_cap));
    *n_out = n;
    return copy_out(e, out, e->V.ex_rec, sizeof(cph_exchange_record) * n, stream);
}
int64_t cph_get_step(const cph_engine* e) { return e ? e->h_step : -1; }
int cph_set_step(cph_engine* e, int64_t step) {
    if (!e || step < 0) return fail(e, CPH_E_INVALID, "bad arguments");
    long long s = step;
    TRY(copy_in(e, e->V.step, &s, sizeof s, nullptr));
    e->h_step = step;
    return CPH_OK;
}
// ---- checkpoint: one host byte buffer, header then fixed-order sections
namespace {
struct CkHeader {
    char magic[8];
    uint32_t version;
    int32_t W, total_atoms, site_rows;
    uint64_t seed;
    int64_t step;
};
constexpr uint32_t kCkVersion = 1;

struct CkLayout {
    size_t x, v, st, slot, wat, vs, ex, stats, occ, vis, nobs, total;
};

CkLayout ck_layout(const cph_engine* e) {
    const size_t W = e->V.W, N = e->V.total_atoms, S = e->h_w_site_off.back();
    CkLayout L;
    size_t o = sizeof(CkHeader);
    auto take = [&o](size_t bytes) { const size_t at = o; o += (bytes + 7) & ~size_t(7); return at; };
    L.x = take(3 * N * sizeof(double));
    L.v = take(3 * N * sizeof(double));
    L.st = take(S * sizeof(int));
    L.slot = take(W * sizeof(int));
    L.wat = take(W * sizeof(int));
    L.vs = take(W * sizeof(double));
    L.ex = take(4 * sizeof(int));
    L.stats = take(10 * sizeof(long long));
    L.occ = take(S * CPH_MAX_STATES * sizeof(long long));
    L.vis = take(W * W * sizeof(long long));
    L.nobs = take(sizeof(long long));
    L.total = o;
    return L;
}
} // namespace

size_t cph_state_bytes(const cph_engine* e) { return e ? ck_layout(e).total : 0; }

int cph_get_state(cph_engine* e, void* buf, size_t bytes, void* stream) {
    if (!e || !buf) return fail(e, CPH_E_INVALID, "NULL argument");
    const CkLayout L = ck_layout(e);
    if (bytes < L.total) return fail(e, CPH_E_INVALID, "state buffer holds %zu bytes, %zu needed", bytes, L.total);
    char* b = (char*)buf;
    const size_t W = e->V.W, N = e->V.total_atoms, S = e->h_w_site_off.back();
    CkHeader h{};
    memcpy(h.magic, "CPHCKPT", 8);
    h.version = kCkVersion;
    h.W = (int32_t)W;
    h.total_atoms = (int32_t)N;
    h.site_rows = (int32_t)S;
    h.seed = e->V.seed;
    h.step = e->h_step;
    memcpy(b, &h, sizeof h);
    TRY(copy_out(e, b + L.x, e->V.x, 3 * N * sizeof(double), stream));
    TRY(copy_out(e, b + L.v, e->V.v, 3 * N * sizeof(double), stream));
    if (S) TRY(copy_out(e, b + L.st, e->V.site_state, S * sizeof(int), stream));
    TRY(copy_out(e, b + L.slot, e->V.slot_of, W * sizeof(int), stream));
    TRY(copy_out(e, b + L.wat, e->V.walker_at, W * sizeof(int), stream));
    TRY(copy_out(e, b + L.vs, e->V.vscale, W * sizeof(double), stream));
    TRY(copy_out(e, b + L.ex, e->V.ex_state, 4 * sizeof(int), stream));
    TRY(copy_out(e, b + L.stats, e->V.stats, 10 * sizeof(long long), stream));
    if (S) TRY(copy_out(e, b + L.occ, e->V.occ, S * CPH_MAX_STATES * sizeof(long long), stream));
    TRY(copy_out(e, b + L.vis, e->V.visits, W * W * sizeof(long long), stream));
    TRY(copy_out(e, b + L.nobs, e->V.n_obs, sizeof(long long), stream));
    return CPH_OK;
}

int cph_set_state(cph_engine* e, const void* buf, size_t bytes, void* stream) {
    if (!e || !buf) return fail(e, CPH_E_INVALID, "NULL argument");
    const CkLayout L = ck_layout(e);
    const char* b = (const char*)buf;
    const size_t W = e->V.W, N = e->V.total_atoms, S = e->h_w_site_off.back();
    CkHeader h;
    if (bytes < sizeof h) return fail(e, CPH_E_INVALID, "state buffer too short");
    memcpy(&h, b, sizeof h);
    if (memcmp(h.magic, "CPHCKPT", 8) != 0 || h.version != kCkVersion)
        return fail(e, CPH_E_INVALID, "not an engine checkpoint (or another version)");
    if ((size_t)h.W != W || (size_t)h.total_atoms != N || (size_t)h.site_rows != S || bytes < L.total)
        return fail(e, CPH_E_INVALID, "checkpoint of another layout: %d walkers, %d atoms, %d site rows",
                    h.W, h.total_atoms, h.site_rows);
    if (h.step < 0) return fail(e, CPH_E_INVALID, "negative step in checkpoint");
    const double* x = (const double*)(b + L.x);
    const double* v = (const double*)(b + L.v);
    for (size_t k = 0; k < 3 * N; ++k)
        if (!std::isfinite(x[k]) || !std::isfinite(v[k])) return fail(e, CPH_E_INVALID, "non-finite coordinate in checkpoint");
    std::vector<int> slot((const int*)(b + L.slot), (const int*)(b + L.slot) + W);
    int ex[4];
    memcpy(ex, b + L.ex, sizeof ex);
    for (int k = 0; k < 4; ++k)
        if (ex[k] < 0) return fail(e, CPH_E_INVALID, "bad exchange counters in checkpoint");
    // validated setters: site states (also rebuild the charges) and condition map
    if (S) TRY(cph_set_site_states(e, (const int*)(b + L.st), stream));
    TRY(cph_set_condition_map(e, slot.data(), stream));
    TRY(copy_in(e, e->V.x, x, 3 * N * sizeof(double), stream));
    TRY(copy_in(e, e->V.v, v, 3 * N * sizeof(double), stream));
    TRY(copy_in(e, e->V.vscale, b + L.vs, W * sizeof(double), stream));
    TRY(copy_in(e, e->V.ex_state, ex, sizeof ex, stream));
    TRY(copy_in(e, e->V.stats, b + L.stats, 10 * sizeof(long long), stream));
    if (S) TRY(copy_in(e, e->V.occ, b + L.occ, S * CPH_MAX_STATES * sizeof(long long), stream));
    TRY(copy_in(e, e->V.visits, b + L.vis, W * W * sizeof(long long), stream));
    TRY(copy_in(e, e->V.n_obs, b + L.nobs, sizeof(long long), stream));
    TRY(cph_set_step(e, h.step));
    if (h.seed != e->V.seed) { // captured graphs hold the old key in their kernel parameters
        e->V.seed = h.seed;
        for (auto& g : e->graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
    return CPH_OK;
}

int cph_status(cph_engine* e, void* stream) {
    if (!e) return fail(nullptr, CPH_E_INVALID, "NULL engine");
    int st = 0;
    TRY(copy_out(e, &st, e->V.status, sizeof(int), stream));
    if (st)
        return fail(e, CPH_E_NONFINITE,
                    "non-finite value produced or SHAKE unsettled (flags %d: 1 force, 2 position, 4 pair sum, "
                    "8 SHAKE did not converge)", st);
    return CPH_OK;
}

} // extern "C"
