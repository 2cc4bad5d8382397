// Internal layout shared by the engine's translation units (not part of the ABI).
//
// Device memory layout (SoA over "global atoms"; atom a of walker w is global
// atom w_off[w] + a; per-system parameters are indexed sys_poff[s] + a):
//   x, v, F, Fd      double [3 * total_atoms]   xyz interleaved
//   q                double [total_atoms]        current charges (MC changes them)
//   psi, R, dRdpsi   double [total_atoms]        Born-radius pass results
//   c                double [total_atoms]        dE/dR dR/dpsi rt/2 (chain-rule weights)
//   rho, rt, sc      double [system atoms]       intrinsic radius, rho - offset, screen*rt
//   sigh, sqe, mass  double [system atoms]       sigma/2, sqrt(eps), mass
//   eacc             int64  [W * 5]              fixed-point (2^32) energy terms per walker
//   Ffix, dRfix      int64  [3N], [N]            fixed-point (2^32) pair-force and dE/dR sums
//   xs, gq           float4 [total_atoms]        FP32 positions / GB terms for the pair kernels
//   c32              float  [total_atoms]        FP32 chain-rule weights
//   pb32, plj32      float4, float2 [system atoms] static FP32 radii / LJ parameters
//   occ              int64  [sites * 8]          state counts per (slot, site) row
//   visits           int64  [W * W]              samples per (walker, slot)
#pragma once
#include <cstdint>
#include "../../include/cphremd.h"

namespace cph {

struct Item {
    int w;  // walker
    int i0; // first atom of the i-tile
    int st; // (system, i-tile) index into the masked-tile table
    int pad;
};

struct View {
    // walkers
    int W, total_atoms;
    const int* w_sys;
    const int* w_off;
    const int* a_walker;
    const int* w_site_off;
    // systems
    const int* sys_n;
    const int* sys_poff;
    const int* sys_site_off;
    const double *rho, *rt, *sc, *sigh, *sqe, *mass;
    const double *irt, *irho; // 1/rt and 1/rho per system atom (no FP64 division per step)
    const int *excl_off, *excl_j;
    const int *bond_off, *bond_idx, *bond_ij;
    const double *bond_k, *bond_r0;
    const int *ang_off, *ang_idx, *ang_ijk;
    const int *sys_bond_off, *sys_ang_off; // per-system ranges of the bond / angle arrays
    const long long* w_tf_off;             // per-walker offset into tforce (floats)
    float* tforce;                         // per-term bonded forces: bonds [2][3], angles [3][3]
    const double *ang_k, *ang_t0;
    const double2* ang_cs0;                // (cos theta0, sin theta0) per angle
    const int *mt_off, *mt_list;
    // sites (global site index g = sys_site_off[s] + k)
    const int *site_kind, *site_nat, *site_aoff, *site_atoms, *site_nst, *site_qoff, *site_noff;
    const double* site_q;
    const int *site_np, *site_ne;
    const double *site_ref, *site_uref;
    // dynamic state
    double *x, *v, *q, *psi, *R, *dRdpsi, *c, *Fd, *F;
    long long *Ffix, *dRfix, *Hfix; // FP32 symmetric passes: fixed-point force, dE/dR, descreening sums
    const int *smt_off, *smt_list; // masked 32-atom j-tiles per (system, 256-atom i-tile)
    long long* eacc;
    int *slot_of, *walker_at, *site_state;
    double* vscale;
    long long* step;
    int* status;
    int* ex_state; // [0] exchange events, [1..3] attempts along E, pH, T
    long long* stats; // [10]
    cph_mc_record* mc_rec;
    // MC sweep scratch per (walker, site): proposal, ln u, dU at the sweep's
    // start charges, and whether the sweep accepted it
    int *mc_from, *mc_to, *mc_take;
    double *mc_lnu, *mc_du0;
    cph_exchange_record* ex_rec;
    int* ex_n;
    // sampling observables: per (slot, site) state counts, per (walker, slot) visits, samples
    long long *occ, *visits, *n_obs;
    // grid
    const double *gE, *gpH, *gT;
    int nE, npH, nT, n_order;
    int order[3];
    // parameters
    double tau, inv_eps_in, sqrt_k, alpha, beta, gamma, offset, dt, gamma_ln;
    // Langevin factors: (1 - g dt/2), 1 / (1 + g dt/2), per system atom
    // dt A / m and sqrt(2 g kB A dt / m), per temperature sqrt(T)
    double lg_c1, lg_c2;
    const double *lg_im, *lg_sf, *lg_sqT;
    // salt screening: kappa (1/A), 1/eps_out, and the factor the finishing
    // kernels apply to pair sums (tau without salt; 1 with salt, whose pair
    // kernels carry tau(f) per pair)
    double kappa, inv_eps_out, tau_pair;
    // the FP32 GB and MC kernels' copies of tau, 1/eps_in, 1/eps_out, kappa and
    // sqrt(k), rounded once on the host: a kernel that reloads one of them
    // under register pressure then reads a parameter instead of converting the
    // double again (a conversion issues to the narrow FP64 pipe)
    float tau32, iei32, ieo32, kappa32, sqk32;
    double sa_gamma, sa_probe; // nonpolar surface term (ACE), 0 = off
    // SHAKE: clusters (one heavy atom and its hydrogens) per system, work
    // items (walker, cluster), positions before the Langevin step
    const int *shk_heavy, *shk_off, *shk_h, *shk_item_w, *shk_item_c;
    const double* shk_d;
    double* xprev; // null when SHAKE is off
    double shake_tol;
    float rfar2; // pairs with r^2 >= rfar2 are in the series regime in both directions
    float smax32; // largest descreening radius s over every system atom
    // Born-radius cutoff (AMBER's rgbmax): descreening shells beyond it do not
    // count; INFINITY = none
    double rgbmax;
    // FP32 pair-kernel operands, staged once per step by one thread per atom
    float4* xs;          // (x, y, z, 0) relative to the walker's first atom
    float4* gq;          // (sqrt(k) q, R, 1/R, log2(e) / (4 R)), after the Born radii and MC
    float* c32;          // chain-rule weights c
    const float4* pb32;  // per system atom, static: (s, rt, 1/rt, 0)
    const float2* plj32; // per system atom, static: (sigma/2, sqrt(eps))
    unsigned long long seed;
    int tex_semigrand; // T exchange on U - sum U_ref + sum_redox F N_e (E - E0_ref) instead of U
    const int* sys_ordered; // per system: 1 = ordered passes (one warp per atom), 0 = symmetric tiles
    // per walker: 1 = advanced by this engine; 0 = kept but not computed (a
    // walker another engine of a sharded grid advances)
    const int* w_local;
    cph_exchange_row* ex_rows; // [W] exchange inputs per walker (this engine's or gathered)
    int first_local;           // lowest local walker (counts the observables' samples)
};

} // namespace cph
