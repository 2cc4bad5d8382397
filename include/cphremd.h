/*
 * cphremd.h -- C ABI of the GB300 engine for multidimensional E,pH,T replica
 * exchange with constant pH and redox potential MD (C(pH,E)MD) in OBC
 * generalized-Born implicit solvent (Cruzeiro & Roitberg, arXiv 1809.07726).
 *
 * Paper passages the calls follow (section names of the paper):
 *   - C(pH,E)MD: MD runs for a set number of steps, then protonation and/or
 *     redox state changes are attempted by Monte Carlo; protonation goes first
 *     when both fall on one step; intervals are independent
 *     ("Constant pH and Redox Potential Molecular Dynamics").
 *   - Exchange probabilities along pH, E and T: eqs (3), (4), (5).
 *   - Multidimensional REMD: one dimension per attempt, in a user order,
 *     between nearest neighbours that share the other two conditions, every
 *     EAF steps ("AMBER's multidimensional REMD module").
 *   - Implicit solvent: the Onufriev-Bashford-Case GB model ("igb=2") is used
 *     for MD and for the state-change attempts ("Implicit Solvent
 *     Calculations"); Langevin dynamics with 10 ps^-1 friction and 2 fs steps
 *     (same section).
 *
 * Conventions
 *   Units: kcal/mol, Angstrom, e, amu, ps, K, V.
 *   Every call returns CPH_OK (0) or a negative CPH_E_* code; the message of
 *   the last failure is available from cph_last_error().  No C++ exception
 *   crosses this interface.  Calls on one engine are not thread-safe.
 *   Host pointers ("host") are read during the call and not retained; device
 *   pointers ("device") belong to the caller.  The engine owns every device
 *   buffer it allocates; cph_destroy() frees them.
 *   Work on an engine is queued on the CUDA stream passed as `stream`
 *   (a cudaStream_t; NULL = the legacy default stream).  Getters synchronise
 *   that stream first.  Asynchronous device errors surface at the next getter
 *   or cph_status().
 *
 * Condition grid: slot = iE + nE * (ipH + npH * iT).  Walker w starts at slot
 * w; exchanges move walkers between slots (conditions), never coordinates.
 * Atom a of walker w is stored at global index offsets[w] + a
 * (cph_walker_offsets).
 */
#ifndef CPHREMD_H
#define CPHREMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes */
#define CPH_OK 0
#define CPH_E_INVALID (-1)   /* bad argument or descriptor; nothing was changed */
#define CPH_E_CUDA (-2)      /* a CUDA runtime call failed */
#define CPH_E_OOM (-3)       /* device allocation failed */
#define CPH_E_NONFINITE (-4) /* a non-finite force, energy or position was produced */
#define CPH_E_TIMEOUT (-5)   /* a bounded device-side wait gave up */
#define CPH_E_STATE (-6)     /* call not valid in the engine's current state */

/* ---- enumerations */
#define CPH_SITE_PH 0
#define CPH_SITE_REDOX 1

#define CPH_DIM_E 0
#define CPH_DIM_PH 1
#define CPH_DIM_T 2
#define CPH_DIM_NEXT (-1) /* next dimension of the user order */

#define CPH_MC_PH 1
#define CPH_MC_REDOX 2
#define CPH_MC_BOTH 3 /* protonation sweep, then redox sweep */

#define CPH_PREC_FP64 0 /* FP64 pair arithmetic and accumulation */
#define CPH_PREC_FP32 1 /* FP32 pair arithmetic, int64 fixed-point accumulation */

/* energy terms returned per walker */
#define CPH_E_GB 0
#define CPH_E_COUL 1
#define CPH_E_LJ 2
#define CPH_E_BOND 3
#define CPH_E_ANGLE 4
#define CPH_E_TOTAL 5
#define CPH_NTERMS 6

/* ---- descriptors (all host memory, copied by cph_init_system) */

/* A titratable site ("Constant pH and Redox Potential MD" section): a set of
 * atoms whose charges take one of n_states discrete sets. */
typedef struct cph_site_desc {
    int kind;             /* CPH_SITE_PH or CPH_SITE_REDOX */
    int n_atoms;          /* atoms whose charge changes, 1..64 */
    const int* atoms;     /* [n_atoms] atom indices in the system */
    int n_states;         /* 2..8 */
    const double* q;      /* [n_states * n_atoms] charges, state-major */
    const int* n_prot;    /* [n_states] protons of each state (pH sites) */
    const int* n_elec;    /* [n_states] electrons of each state (redox sites) */
    double ref;           /* pKa_ref (pH site) or E0_ref in volts (redox site) */
    int init_state;       /* starting state */
} cph_site_desc;

/* One molecular system.  Sites must not share atoms.  Exclusions from
 * Coulomb and LJ are every pair one or two bonds apart (1-2 and 1-3 in the
 * bond graph) plus the optional extra list; GB runs over all pairs. */
typedef struct cph_system_desc {
    int n_atoms;                    /* 1..65536 */
    const double* x;                /* [3N] starting positions, xyz interleaved */
    const double* v;                /* [3N] starting velocities (A/ps) or NULL for zero */
    const double* mass;             /* [N] amu, > 0 */
    const double* q;                /* [N] charges; site atoms are overwritten by the
                                       charges of the site's init_state */
    const double* rho;              /* [N] intrinsic Born radii (A), > gb.offset */
    const double* screen;           /* [N] HCT screening factors */
    const double* sigma;            /* [N] LJ sigma (A); Lorentz-Berthelot mixing */
    const double* eps;              /* [N] LJ epsilon (kcal/mol) */
    int n_bonds;
    const int* bonds;               /* [2 * n_bonds] atom pairs */
    const double* bond_k;           /* [n_bonds] E = k (r - r0)^2 */
    const double* bond_r0;          /* [n_bonds] */
    int n_angles;
    const int* angles;              /* [3 * n_angles] i-j-k, j the vertex */
    const double* angle_k;          /* [n_angles] E = k (theta - theta0)^2 */
    const double* angle_t0;         /* [n_angles] radians */
    int n_excl;
    const int* excl;                /* [2 * n_excl] extra excluded pairs, or NULL */
    int n_sites;
    const cph_site_desc* sites;     /* [n_sites]; swept in index order within a kind */
} cph_system_desc;

/* The E x pH x T grid ("AMBER's multidimensional REMD module"). */
typedef struct cph_grid_desc {
    int nE, npH, nT;                /* each >= 1 */
    const double* E;                /* [nE] volts, ascending */
    const double* pH;               /* [npH] ascending */
    const double* T;                /* [nT] kelvin, ascending */
    const int* system_of_slot;      /* [nE*npH*nT] system index of the walker starting there */
    int n_order;                    /* 1..3 */
    int order[3];                   /* exchange dimension order, CPH_DIM_* */
} cph_grid_desc;

/* OBC generalized-Born parameters ("igb=2": offset 0.09 A, alpha 0.8,
 * beta 0.0, gamma 2.909125; eps_in 1, eps_out 78.5; "igb=5" is alpha 1.0,
 * beta 0.8, gamma 4.85).  kappa >= 0 (1/A) screens the solvent reaction field
 * by salt in the Debye-Hueckel form: every GB term -k q_i q_j tau / f takes
 * tau(f) = 1/eps_in - exp(-kappa f)/eps_out (f = R for the self terms); the
 * paper states no salt, and 0 (the default) gives the constant
 * 1/eps_in - 1/eps_out.  The differentiable energy (cph_gb_energy*) takes
 * every option: salt, the surface term and the cutoff. */
typedef struct cph_gb_params {
    double eps_in, eps_out;
    double offset;                  /* rho_tilde = rho - offset */
    double alpha, beta, gamma;      /* tanh(alpha psi - beta psi^2 + gamma psi^3) */
    double kappa;                   /* salt screening, 1/A (0 = none) */
    /* nonpolar surface term in the ACE approximation (Schaefer & Karplus),
     * reported with E_GB: sum_i 4 pi sa_gamma (rho_i + sa_probe)^2
     * (rho_i / R_i)^6; sa_gamma in kcal/mol/A^2 (0 = off, e.g. 0.005),
     * sa_probe in A (e.g. 1.4) */
    double sa_gamma, sa_probe;
    /* Born-radius cutoff in A (AMBER's rgbmax; 0 = none): only descreening
     * shells at distance t <= rgbmax from an atom count in its OBC integral
     * sum psi, i.e. the HCT integrals run to min(r + s, rgbmax) and
     * the fully covered shells of a ball inside a sphere end at rgbmax.
     * Finite and >= 0, else CPH_E_INVALID. */
    double rgbmax;
} cph_gb_params;

typedef struct cph_run_params {
    cph_gb_params gb;
    double dt;                      /* ps, e.g. 0.002 */
    double gamma_ln;                /* Langevin friction, ps^-1, e.g. 10 */
    int precision;                  /* CPH_PREC_FP64 or CPH_PREC_FP32 */
    int mc_ph_every;                /* protonation sweep interval in steps (0 = never) */
    int mc_redox_every;             /* redox sweep interval in steps (0 = never) */
    int exchange_every;             /* steps between exchange attempts (0 = never) */
    /* SHAKE (Implicit Solvent Calculations section: 2 fs steps with the
     * lengths of all bonds to hydrogen constrained).  1: after every Langevin
     * step, each bond that involves an atom lighter than 2 amu is held at its
     * r0 by SHAKE (iterated along the old bond vectors until
     * |r0^2 - r^2| <= 2 shake_tol r0^2; velocities take the displacement / dt),
     * and those bonds' harmonic terms are left out.  A bond between two such
     * atoms, or more than 8 on one heavy atom, is refused.  0: no
     * constraints. */
    int shake;
    double shake_tol;               /* > 0 when shake = 1, e.g. 1e-8 */
    /* Energy eps of the T exchange, eq (5) ("the energy of the system"):
     * CPH_TEX_POTENTIAL (0, default): the total potential energy U.
     * CPH_TEX_SEMIGRAND (1): U - sum_k U_ref,k(s_k)
     *   + sum_{redox k} F N_e,k(s_k) (E - E0_ref,k), the part of the C(pH,E)MD
     *   weight exp(-G/kT) that scales with 1/kT (G the state free energy of the
     *   MC moves with U_el completed to U; the pH term does not scale with T).
     *   With it one T attempt is in detailed balance with the C(pH,E)MD
     *   ensemble of each walker's states; the two differ only when the pair's
     *   site states differ.  Other values: CPH_E_INVALID. */
    int t_exchange_energy;
} cph_run_params;

#define CPH_TEX_POTENTIAL 0
#define CPH_TEX_SEMIGRAND 1

typedef struct cph_engine cph_engine; /* opaque */

/* One Monte-Carlo decision of the last cph_mc_titrate / cph_run MC event. */
typedef struct cph_mc_record {
    int walker, site, from, to, accepted, pad_;
    double dU;      /* U_el(to) - U_el(from), kcal/mol */
    double x;       /* -(G(to) - G(from)) / kT */
    double lnu;     /* ln u of the acceptance draw; accepted = lnu < x */
} cph_mc_record;

/* One pair of the last exchange attempt. */
typedef struct cph_exchange_record {
    int dim, slot_lo, slot_hi, walker_lo, walker_hi, accepted;
    double x;       /* exponent of eq (3), (4) or (5) */
    double lnu;
} cph_exchange_record;

/* ---- engine lifetime */

/* Validate the descriptors, compute each site state's isolated reference
 * energy U_ref (U_el of the site's atoms alone in the starting geometry),
 * allocate device state for every walker of the grid and upload it.
 * Random numbers come from Philox4x32-10 keyed by `seed`.  On failure *out is
 * NULL and cph_last_error(NULL) describes why. */
int cph_init_system(const cph_system_desc* sys, int n_sys, const cph_grid_desc* grid,
                    const cph_run_params* p, uint64_t seed, cph_engine** out);
void cph_destroy(cph_engine* e);
/* Message of the last failure on `e`, or of the calling thread's last failed
 * cph_init_system / ABI-level call when e is NULL.  Never NULL. */
const char* cph_last_error(const cph_engine* e);

int cph_num_walkers(const cph_engine* e);
int cph_total_atoms(const cph_engine* e);
int cph_walker_offsets(const cph_engine* e, int* offsets /* host [W+1] */);
int cph_site_offsets(const cph_engine* e, int* offsets /* host [W+1] into site-state arrays */);

/* ---- the hot path */

/* Launch shape of the hot path: CPH_LAUNCH_BATCHED (default) runs every
 * walker of the grid in one launch per pass; CPH_LAUNCH_PER_REPLICA issues the
 * same kernels once per walker (the one-replica-per-process shape of the
 * paper's runs), for comparison.  Results are bitwise identical. */
#define CPH_LAUNCH_BATCHED 0
#define CPH_LAUNCH_PER_REPLICA 1
int cph_set_launch_mode(cph_engine* e, int mode);
/* Streams of the per-replica launch mode: walker w's launches go to internal
 * stream w mod n (n = 1..32; 1, the default, keeps them on the caller's
 * stream).  Each per-walker launch sequence is forked from the caller's
 * stream and joined back to it, as one process per replica sharing a GPU
 * would overlap.  Results are bitwise identical for any n. */
int cph_set_replica_streams(cph_engine* e, int n);

/* Forces and energies of every walker at the current state (Born radii,
 * GB + Coulomb + LJ pair pass, chain rule through the radii, bonded terms,
 * energy totals); nothing moves. */
int cph_evaluate(cph_engine* e, void* stream);
/* n_steps of plain MD (no MC, no exchange) for every walker; the step counter
 * advances by n_steps. */
int cph_step_replicas(cph_engine* e, int64_t n_steps, void* stream);
/* One Monte-Carlo sweep at the current positions: kind = CPH_MC_PH, REDOX or
 * BOTH (protonation first).  Each sweep visits every site of that kind once,
 * in index order, proposing a uniformly chosen other state and accepting with
 * the Metropolis rule on G(s) = U_el(s) - U_ref(s) + kT ln10 N_H(s)(pH - pKa_ref)
 * + F N_e(s)(E - E0_ref) at fixed Born radii. */
int cph_mc_titrate(cph_engine* e, int kind, void* stream);
/* One exchange attempt along `dim` (CPH_DIM_E/PH/T, or CPH_DIM_NEXT for the
 * next dimension of the order).  Neighbours (m, m+1) of the attempt's parity
 * (alternating per dimension) within each line of the other two conditions,
 * walkers of the same system only; accept iff ln u < x with x from eq (3),
 * (4) or (5); T swaps scale velocities by sqrt(T_new/T_old).  A T attempt
 * evaluates the energies at the current state first. */
int cph_attempt_exchanges(cph_engine* e, int dim, void* stream);
/* n_steps of the full schedule.  Step t: Born radii at x_t; protonation sweep
 * if t > 0 and t % mc_ph_every == 0; redox sweep if t > 0 and
 * t % mc_redox_every == 0; pair pass and bonded terms; exchange along the next
 * dimension if t > 0 and t % exchange_every == 0; Langevin step to x_{t+1}.
 * Whole periods of the schedule replay a captured CUDA graph. */
int cph_run(cph_engine* e, int64_t n_steps, void* stream);

/* Tile shape of a system's pair passes in FP32 mode (FP64 mode always runs
 * the ordered form):
 *   CPH_SHAPE_SYMMETRIC (default): every unordered pair once, a CTA of 128
 *     threads owning a 256-atom i-tile against chunks of 32-atom j-tiles, both
 *     atoms' sums in int64 fixed point (best for large systems);
 *   CPH_SHAPE_WARP_PER_ATOM: every ordered pair, one warp per atom i with its
 *     lanes over j and a fixed-order warp reduction; twice the pair arithmetic
 *     but 64 times more CTAs, for systems too small to fill the GPU with
 *     256-atom tiles.
 * Both forms meet the same accuracy bars; their results differ in the last
 * bits (different summation order), so a run is bitwise reproducible only
 * with the same shapes.  Batched and per-replica launches agree bitwise for
 * any shapes.  CPH_E_INVALID for a bad system index or shape. */
#define CPH_SHAPE_SYMMETRIC 0
#define CPH_SHAPE_WARP_PER_ATOM 1
int cph_set_tile_shape(cph_engine* e, int system, int shape);
int cph_get_tile_shapes(const cph_engine* e, int* shapes /* host [n_sys] */);

/* ---- one replica grid sharded over several engines (one per GPU)
 *
 * Walkers are independent between exchanges ("AMBER's multidimensional REMD
 * module" exchanges only conditions between replicas), so a grid can be split
 * by walker over several engines, each built from the same systems, grid,
 * parameters and seed on its own GPU: cph_set_local_walkers gives each the
 * walkers it advances (the others are kept but not computed).  Every random
 * number is keyed by the global walker, site and slot, so the sharded run is
 * bitwise the single-engine run.  At an exchange step t (t > 0, t a multiple
 * of exchange_every) the host of each engine:
 *   1. cph_mc_titrate for the MC kinds due at t (Born radii at x_t, sweeps);
 *   2. cph_exchange_rows: energies at x_t, then one row per local walker;
 *   3. gathers the rows of all engines (any transport, e.g. an all-gather);
 *   4. cph_exchange_apply with every walker's row: the same attempt, on the
 *      same rows and random numbers, on every engine; it updates the condition
 *      map and scales the local walkers' velocities after a T swap;
 *   5. cph_step_replicas(e, 1): the MD step t.
 * Other steps run through cph_run, which refuses (CPH_E_STATE, nothing
 * launched) a span that holds an exchange step on a sharded engine; so does
 * cph_attempt_exchanges.  Observables count local walkers only (sum the
 * counts over the engines); getters of per-walker state are meaningful for
 * local walkers only. */
typedef struct cph_exchange_row {
    int walker;           /* global walker index */
    int n_prot, n_elec;   /* N_H and N_e of its current site states */
    int pad_;
    long long u_fix;      /* total potential energy at x_t, fixed point (2^-32 kcal/mol units) */
    double uref_sum;      /* sum over its sites of U_ref(state), kcal/mol */
    double e0ref_ne_sum;  /* sum over its redox sites of N_e(state) E0_ref, V */
} cph_exchange_row;
/* walkers: host [n] distinct global walker indices (n = W: all, the default).
 * Drops captured graphs; the engine's state is otherwise unchanged. */
int cph_set_local_walkers(cph_engine* e, int n, const int* walkers);
/* Energies at the current state of the local walkers, then their rows into
 * rows (host, max entries); *n_out = the number of local walkers.
 * Synchronises `stream`.  CPH_E_INVALID if max is too small. */
int cph_exchange_rows(cph_engine* e, cph_exchange_row* rows, int max, int* n_out, void* stream);
/* One exchange attempt along `dim` (as cph_attempt_exchanges) on the rows of
 * all W walkers (host, any order, each walker exactly once; CPH_E_INVALID
 * otherwise, nothing launched). */
int cph_exchange_apply(cph_engine* e, int dim, const cph_exchange_row* rows, int n_rows, void* stream);

/* Diagnostic timing of the three pair passes at the current state, with CUDA
 * events recorded on `stream` around each launch (batched or per-replica, per
 * the launch mode): ms[0] Born radii, ms[1] GB + Coulomb + LJ, ms[2] chain
 * rule + bonded terms, each the mean over `reps` launches.  The passes only
 * rewrite derived per-atom quantities (radii, forces); positions, velocities,
 * charges and site states are unchanged.  Synchronises `stream`. */
int cph_time_passes(cph_engine* e, int reps, double* ms /* host [3] */, void* stream);

/* Diagnostic for the roofline of the pair passes: throughput of the FP32 (FMA)
 * pipe, driven by packed f32x2 FMAs, and of the MUFU pipe, driven by
 * rsqrt.approx, on the current device, timed with CUDA events on `stream`
 * (best of three runs of about a millisecond each, after one warm-up run).
 * Outputs are operations per second over the whole GPU (an FMA counts once);
 * divided by the SM count and the SM clock they give the per-SM rates the
 * roofline uses.  Allocates nothing; synchronises `stream`. */
int cph_probe_pipe_rates(double* fp32_ops_per_s, double* mufu_ops_per_s, void* stream);

/* Tile-shape autotuner (FP32 mode): times the three pair passes at the
 * current state for each candidate and keeps the fastest.  First the
 * symmetric work-item size (j-tiles of 32 atoms per CTA: 8..128; results of
 * later steps are bitwise the same whatever size is chosen, fixed-point
 * sums); then the per-system tile shape: systems of at most n atoms run
 * CPH_SHAPE_WARP_PER_ATOM, the others CPH_SHAPE_SYMMETRIC, for n over the
 * distinct system sizes and 0 (every system symmetric).  *chosen (may be
 * NULL) receives the work-item size; cph_get_tile_shapes reports the shapes.
 * A change of shape changes later results in the last bits (see
 * cph_set_tile_shape).  Derived per-atom quantities are rewritten as by
 * cph_time_passes.  FP64 mode has nothing to tune (*chosen = 0).
 * Synchronises `stream`. */
int cph_autotune(cph_engine* e, void* stream, int* chosen);

/* ---- getters and setters (host buffers; getters synchronise `stream`) */
int cph_get_energies(cph_engine* e, double* out /* [W * CPH_NTERMS] */, void* stream);
int cph_get_forces(cph_engine* e, double* out /* [total_atoms * 3] */, void* stream);
int cph_get_born_radii(cph_engine* e, double* out /* [total_atoms] */, void* stream);
int cph_get_positions(cph_engine* e, double* out /* [total_atoms * 3] */, void* stream);
int cph_set_positions(cph_engine* e, const double* in, void* stream);
int cph_get_velocities(cph_engine* e, double* out, void* stream);
int cph_set_velocities(cph_engine* e, const double* in, void* stream);
int cph_get_charges(cph_engine* e, double* out /* [total_atoms] */, void* stream);
int cph_get_site_states(cph_engine* e, int* out /* [site_offsets[W]] */, void* stream);
int cph_set_site_states(cph_engine* e, const int* in, void* stream); /* also resets charges */
int cph_get_counts(cph_engine* e, int* n_prot, int* n_elec /* [W] each */, void* stream);
int cph_get_condition_map(cph_engine* e, int* slot_of_walker /* [W] */, void* stream);
int cph_set_condition_map(cph_engine* e, const int* slot_of_walker, void* stream);
/* [0..5]: exchange attempts / accepted pairs along E, pH, T (pairs tried and
 * pairs swapped); [6..9]: MC proposals / acceptances for pH, redox sites. */
int cph_get_accept_stats(cph_engine* e, int64_t* out /* [10] */, void* stream);
int cph_get_reference_energies(cph_engine* e, double* out /* [sum over systems of
                               sum over sites of n_states] */);
/* Records of the last MC event: one per (walker, visited site), walker-major. */
int cph_get_mc_records(cph_engine* e, cph_mc_record* out, int max, int* n_out, void* stream);
int cph_get_exchange_records(cph_engine* e, cph_exchange_record* out, int max, int* n_out,
                             void* stream);
int64_t cph_get_step(const cph_engine* e);
int cph_set_step(cph_engine* e, int64_t step);

/* Checkpoint and restart.  cph_get_state writes into one host buffer of
 * cph_state_bytes(e) bytes everything that, with the engine's systems, grid
 * and run parameters, fixes the rest of the trajectory: positions,
 * velocities, site states, the condition map, the step counter, the Philox
 * seed, the exchange counters (which dimension and which neighbour parity
 * come next), pending velocity scales, the acceptance statistics and the
 * sampling observables.  cph_set_state restores it into an engine built from
 * the same systems, grid and run parameters (any seed: the checkpoint's seed
 * is adopted); the continued run is then bitwise the run that wrote it.  A
 * checkpoint of another layout or version is refused with CPH_E_INVALID and
 * leaves the engine unchanged.  Forces, energies, Born radii and the records
 * of the last MC / exchange event are derived and are not stored.  The
 * buffer's format is private to the library (same version, same build). */
size_t cph_state_bytes(const cph_engine* e);
int cph_get_state(cph_engine* e, void* buf, size_t bytes, void* stream);
int cph_set_state(cph_engine* e, const void* buf, size_t bytes, void* stream);
/* Synchronise `stream` and report device-side status: CPH_OK, CPH_E_NONFINITE
 * (a walker produced a non-finite energy or position) or a CUDA error. */
int cph_status(cph_engine* e, void* stream);
/* Energies returned by cph_get_energies are those of the last evaluation that
 * computed them: cph_evaluate, cph_attempt_exchanges, or a cph_run step that
 * attempted an exchange. */

/* ---- sampling observables
 *
 * The analysis of the "E,pH-REMD at 300 K" results fits E0 with eq (2) to the
 * cumulative fraction of reduced species at every (E, pH) condition, and
 * Figure 7 counts how long each replica spent at every (E, T, pH)
 * combination.  The engine accumulates both on the device: every MD step
 * (cph_run and cph_step_replicas) takes one sample after the step's MC sweeps
 * and exchange attempt, i.e. with the charges and condition the step's
 * dynamics then runs at.
 *
 * Occupancy rows: condition slot s holds, at any time, a walker of system
 * system_of_slot[s] (exchanges never mix systems), so row
 * cph_site_offsets()[s] + k counts the samples in which site k of the walker
 * at slot s was in each state, CPH_MAX_STATES int64 columns per row (columns
 * >= the site's n_states stay 0).  Every row sums to the sample count.
 * Visits: [W * W] int64, walker-major: visits[w * W + s] = samples in which
 * walker w sat at slot s; every row and every column sums to the sample
 * count.  Counts are exact integers, independent of launch shape. */
#define CPH_MAX_STATES 8
int cph_get_occupancy(cph_engine* e, int64_t* out /* [site_offsets[W] * CPH_MAX_STATES] */,
                      int64_t* n_samples /* may be NULL */, void* stream);
int cph_get_visits(cph_engine* e, int64_t* out /* [W * W] */, void* stream);
/* Per occupancy row: the sampled fraction protonated (pH site) or reduced
 * (redox site), sum_state count(state) * (n(state) - n_min) / (n_max - n_min)
 * / n_samples with n = protons (pH) or electrons (redox) of each state; a
 * site whose states all carry the same n gives 0.  CPH_E_STATE when no
 * sample has been taken yet. */
int cph_get_fractions(cph_engine* e, double* out /* [site_offsets[W]] */, void* stream);
/* Zero the occupancy, the visits and the sample count (starts a new
 * accumulation window, e.g. after equilibration). */
int cph_reset_observables(cph_engine* e, void* stream);

/* Least-squares Hill fit of a titration curve (host only, no GPU needed):
 * minimises sum_i (f_i - f(x_i))^2 over (x0, n_hill) with
 *   CPH_FIT_PH:    eq (1), f(pH) = 1 / (1 + 10^(n_hill (pH - pKa))), x0 = pKa;
 *   CPH_FIT_REDOX: eq (2), f(E) = 1 / (1 + exp(n_hill v F (E - E0) / (kB T))),
 *                  x0 = E0 in volts, v electrons, T kelvin.
 * x[n_pts], f[n_pts] host arrays, 0 <= f <= 1.  Started from the linear Hill
 * plot regression, refined by Levenberg-Marquardt.  *rss (may be NULL) gets
 * the residual sum of squares.  CPH_E_INVALID for fewer than two distinct x,
 * f outside [0, 1], a curve with no value strictly inside (0, 1), T <= 0 or
 * v <= 0 (redox), or no convergence in 500 iterations. */
#define CPH_FIT_PH 1
#define CPH_FIT_REDOX 2
int cph_fit_hill(int kind, int n_pts, const double* x, const double* f, double T, double v,
                 double* x0, double* n_hill, double* rss);

/* Predictions of eqs (6)-(8) (host only, no GPU needed).  The "Temperature
 * dependence in predicting E0 vs pH and pKa vs redox potential" section draws
 * Figure 6's solid lines from eqs (7) and (8) with parameters taken from the
 * simulation, without fitting.  A redox-active group (v electrons) couples to
 * n_sites pH-active groups: pka_red[i] / pka_oxi[i] (host [n_sites]) are site
 * i's pKa with the redox group reduced / oxidised; e0_prot / e0_deprot (V) are
 * the redox group's E0 with every pH site protonated / deprotonated; T in K.
 *   eq (6): *delta_e0 = E0_prot - E0_deprot
 *                     = kB T ln10 sum_i (pka_red[i] - pka_oxi[i]) / (v F)
 *   eq (7): e0[k] = E0_prot + kB T / (v F) sum_i ln((10^-pka_red[i] + 10^-pH[k])
 *                                                   / (10^-pka_oxi[i] + 10^-pH[k]))
 *   eq (8): sum_pka[k] = sum_i pka_red[i] + log10((exp(-v F e0_prot / kB T)
 *                        + exp(-F E[k] / kB T)) / (exp(-v F e0_deprot / kB T)
 *                        + exp(-F E[k] / kB T)))
 * The logarithm of eq (8) is read as base 10, and v multiplies only the E0
 * terms, as printed.  pH[n_pts], E[n_pts] (V) host inputs; e0[n_pts],
 * sum_pka[n_pts] host outputs.  CPH_E_INVALID for negative counts, NULL
 * arrays of positive length, T <= 0, v <= 0 or non-finite inputs; nothing is
 * written then. */
int cph_predict_delta_e0(int n_sites, const double* pka_red, const double* pka_oxi, double T,
                         double v, double* delta_e0);
int cph_predict_e0(int n_pts, const double* pH, double e0_prot, int n_sites,
                   const double* pka_red, const double* pka_oxi, double T, double v,
                   double* e0);
int cph_predict_sum_pka(int n_pts, const double* E, double e0_prot, double e0_deprot,
                        int n_sites, const double* pka_red, double T, double v,
                        double* sum_pka);

/* ---- differentiable GB energy (device buffers, caller-owned) */

/* E_GB of n_rep independent configurations of one n-atom system (no Coulomb,
 * no LJ; OBC radii as above, all pairs including self terms).
 *   x      device float [n_rep * n * 3]
 *   q      device float [n_rep * n]
 *   rho    device float [n_rep * n] intrinsic radii (> offset)
 *   screen device float [n] screening factors (shared by all replicas)
 *   E      device double [n_rep], written
 * FP32 pair arithmetic, int64 fixed-point accumulation.  Needs
 * cph_gb_workspace_bytes(n_rep, n) bytes of device workspace (caller-owned,
 * 256-byte aligned); the library allocates nothing. */
size_t cph_gb_workspace_bytes(int n_rep, int n);
int cph_gb_energy(int n_rep, int n, const float* x, const float* q, const float* rho,
                  const float* screen, const cph_gb_params* gb, double* E,
                  void* workspace, size_t workspace_bytes, void* stream);
/* Gradient of sum_r dE[r] * E_GB[r] with respect to x, q and rho (the
 * adjoint of cph_gb_energy).  Born radii are recomputed, not stored.
 *   dE     device double [n_rep] upstream gradient
 *   dx     device float [n_rep * n * 3], dq and drho device float [n_rep * n]:
 *          written (not accumulated). */
int cph_gb_energy_backward(int n_rep, int n, const float* x, const float* q,
                           const float* rho, const float* screen, const cph_gb_params* gb,
                           const double* dE, float* dx, float* dq, float* drho,
                           void* workspace, size_t workspace_bytes, void* stream);

/* ---- GB energy without any device allocation
 *
 * Same result as cph_gb_energy, for callers that cannot allocate device
 * memory themselves: plug-ins that run inside a host program which owns the
 * whole device-memory budget, and loops in which the device-wide
 * synchronisation of cudaMalloc / cudaFree is not acceptable.  The caller
 * passes only the inputs and the output (same layout as cph_gb_energy); the
 * scratch lives in a fixed array inside this library.  The paper has no
 * counterpart: this is a deployment variant of the GB energy, not part of the
 * method.
 *
 * Scratch: a file-scope device array of CPH_GB_NOALLOC_SCRATCH_BYTES (12 MiB),
 * reserved on every GPU where the library's kernels are loaded and held until
 * the process exits.  A call needs cph_gb_workspace_bytes(n_rep, n) bytes of
 * it (about 88 bytes per replica-atom: roughly 140,000 replica-atoms, e.g. 17
 * replicas of an 8000-atom system); a larger request returns CPH_E_INVALID
 * and launches nothing.
 * Set-up: the first call on a device looks up the array's device address on
 * that device (the current device at the time of the call); make that first
 * call before any stream capture on that device.
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents (whatever must start at zero is cleared by the kernels).
 * Calls whose work overlaps on the GPU -- on different streams, or from
 * different host threads -- race on the array and corrupt each other's
 * results: serialise them.  No cudaMalloc, cudaFree or other allocating call
 * is made. */
#define CPH_GB_NOALLOC_SCRATCH_BYTES ((size_t)12 << 20)
int cph_gb_energy_noalloc(int n_rep, int n, const float* x, const float* q, const float* rho,
                          const float* screen, const cph_gb_params* gb, double* E, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CPHREMD_H */
