/*
 * bounce.h -- C ABI of the GB300 BOUNCE velocity-jump MD library.
 *
 * Method: Monmarche, Weisman, Lagardere, Piquemal, "BOUNCE: a velocity-jump
 * integrator for molecular dynamics" (arXiv 2002.07109).  The library runs
 * the BJAOAJB splitting of Sec. III.C / Sec. IV.B (BOUNCE) and the BAOAB
 * splitting it extends, for point-charge + Lennard-Jones systems with
 * harmonic bonds and angles, on one CUDA device (sm_103a).
 *
 * Units: Angstrom, fs, kcal/mol, g/mol, elementary charge, K.
 * Coulomb constant 332.063713 kcal A/(mol e^2); k_B = 0.0019872041
 * kcal/(mol K); an acceleration of 1 kcal/mol/A per g/mol is 4.184e-4 A/fs^2.
 *
 * Conventions for every entry point:
 *   - Return value: BOUNCE_OK (0) or a negative BOUNCE_ERR_* code.  Nothing
 *     is thrown across the ABI.  bounce_last_error() returns a message for
 *     the last failing call on that context.  The context stays usable after
 *     an error unless the error is BOUNCE_ERR_CUDA from a sticky device fault.
 *   - Arrays of 3-vectors are row-major (n, 3) doubles.
 *   - Pointer arguments flagged by `where` are host memory (BOUNCE_HOST) or
 *     device memory of the context's device (BOUNCE_DEVICE).  The caller owns
 *     every array it passes; the library copies inputs into its own device
 *     buffers and never keeps a caller pointer after the call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *     of a call is ordered on that stream.  Host-memory transfers through
 *     `where = BOUNCE_HOST` synchronise the stream before returning.
 *   - The F_i of the paper are GRADIENT terms of E_pot (Sec. II.A): the
 *     "gradient" outputs below are dE/dq, not physical forces.
 */
#ifndef BOUNCE_H
#define BOUNCE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BOUNCE_OK 0
#define BOUNCE_ERR_INVALID_ARG (-1)
#define BOUNCE_ERR_CUDA (-2)
#define BOUNCE_ERR_NONFINITE (-3)
#define BOUNCE_ERR_LIST_OVERFLOW (-4)
#define BOUNCE_ERR_STATE (-5)
#define BOUNCE_ERR_UNSUPPORTED (-6)

#define BOUNCE_HOST 0
#define BOUNCE_DEVICE 1

/* Integrators (bounce_run). */
#define BOUNCE_BAOAB 0  /* B A O A B (paper Sec. III.C without J)            */
#define BOUNCE_BOUNCE 1 /* B J A O A J B (paper Sec. III.C and Sec. IV.B)    */
#define BOUNCE_BOUNCE_RESPA 2 /* reciprocal-space kick over Delta/2 = m delta/2
                               * around every block of m BJAOAJB steps (Sec. V) */
#define BOUNCE_BOUNCE_RESPA_EXT 3 /* extended split (Sec. V): the outer kicks add the
                                   * short-range pair part; inner F_0 = bonded only */
#define BOUNCE_BOUNCE_RESPA1 4 /* three levels (Sec. V, RESPA1 splitting): the
                                * reciprocal kick over Delta_out/2 =
                                * respa_m2 respa_m delta/2 around respa_m2
                                * intermediate steps; each kicks with the
                                * short-range pair part over respa_m delta/2
                                * around respa_m BJAOAJB steps with a
                                * bonded-only F_0 */

/* Gradient parts (bounce_compute_gradient). */
#define BOUNCE_GRAD_FULL 0  /* dE_pot/dq: all pairs within r_c + bonded     */
#define BOUNCE_GRAD_SHORT 1 /* F_0: bonded + (1 - chi) W' of every pair     */
#define BOUNCE_GRAD_LONG 2  /* sum_j F_ij = chi W' of every pair (Sec. IV.A) */
#define BOUNCE_GRAD_RECIP 3 /* SPME reciprocal Ewald + same-molecule removal */

#define BOUNCE_MAX_TYPES 4
#define BOUNCE_NOALLOC_MAX_ATOMS 16384

typedef struct bounce_ctx bounce_ctx;

/* Run configuration; bounce_config_default() fills the defaults shown. */
typedef struct bounce_config {
    double dt_fs;          /* time step delta (1.0)                              */
    double gamma_per_fs;   /* Langevin friction gamma (0.001 = 1/ps)             */
    double temperature_K;  /* T (300); beta = 1/(k_B T)                          */
    uint64_t seed;         /* Philox key of every random draw (0)                */
    double r_on;           /* r' : chi = 0 below (4.0); Sec. IV.A                */
    double r_off;          /* r'': chi = 1 above (5.0); r_on == r_off = step     */
    double r_cut;          /* pair cutoff r_c (<= 0 or inf: none)                */
    double skin;           /* Verlet skin; rows hold r < r_c + skin (1.0)        */
    double ewald_beta;     /* 0: bare Coulomb; > 0: Ewald direct erfc (A^-1)     */
    int32_t periodic;      /* 0: open droplet; 1: periodic box                   */
    double box[3];         /* periodic box edges (A)                             */
    int32_t max_neighbors; /* capacity of one candidate row (2048)               */
    int32_t max_short;     /* capacity of one short-range row (256)              */
    int32_t device;        /* CUDA device ordinal (0)                            */
    int32_t pme_grid[3];   /* SPME grid K1 K2 K3; 0 = no reciprocal part (0)     */
    int32_t pme_order;     /* SPME B-spline order, 3..8 (5)                      */
    int32_t respa_m;       /* inner steps per BOUNCE-RESPA outer step, 1..8 (2)  */
    int32_t jump_coulomb;  /* 1: Coulomb is split by chi like LJ (Sec. V droplets);
                            * 0: Coulomb wholly in F_0, only LJ on jumps
                            * (the first example of Sec. IV); with one bound
                            * per type the jump step's rows then keep only
                            * the partners an atom has LJ with (Sec. V: the
                            * partner is drawn among the particles it
                            * interacts with), rebuilt on the displacement of
                            * the types that propose or can be drawn (1)        */
    int32_t pair_bounds;   /* 1: one bound per type pair (Sec. V: L may depend on
                            * the types of both particles) with a two-stage
                            * partner choice: type b with probability
                            * proportional to n_ib Lq_ab (Lq_ab =
                            * ceil(2^16 L_ab / L*_a) + 1, 0 where L_ab = 0),
                            * then uniform within the type; acceptance bound
                            * Lt_ab = Lq_ab L*_a 2^-16.  Rows are then grouped
                            * by partner type (ascending inside each group).
                            * Needs max_neighbors < 65535.  0: one bound L*_a
                            * per atom type, partner uniform over the row (0)  */
    int32_t respa_m2;      /* intermediate steps per BOUNCE-RESPA1 outer step,
                            * 1..8 (3)                                           */
    double pair_skin;      /* skin of the cluster pair lists of the pair sums
                            * (systems with a cutoff); they are rebuilt when an
                            * atom has moved pair_skin/2.  0: the same as skin.
                            * Internal to the pair sums: results do not depend
                            * on it (0)                                         */
    int32_t step_kernel;   /* step kernel: 0 automatic (thread per atom where the
                            * jump bounds predict under 0.5 proposals per
                            * atom-step, else 32-atom cooperative CTAs), 1 the
                            * cooperative kernel, 2 thread per atom (systems
                            * whose pair sums run over clusters or tiles).  Both
                            * give the same results bit for bit (0)            */
} bounce_config;

/* Energies and counters (bounce_get_energies). */
typedef struct bounce_energies {
    double coulomb;     /* sum_{i<j, r<r_c} k q_i q_j / r (or erfc(b r)/r)        */
    double lj;          /* sum_{i<j, r<r_c} 4 eps ((s/r)^12 - (s/r)^6)           */
    double bond;        /* sum k (r - r0)^2                                       */
    double angle;       /* sum k (theta - theta0)^2                               */
    double kinetic;     /* sum m v^2 / 2                                          */
    double potential;   /* coulomb + lj + bond + angle                            */
    double temperature; /* 2 E_kin / (3 N k_B)                                    */
    int64_t step;       /* steps completed since the state was set               */
    int64_t proposals;  /* jump proposals since the last counter reset            */
    int64_t accepts;    /* accepted jumps (reflections)                           */
    int64_t near_ties;  /* proposals with |U - lambda/lambda*| < 1e-6             */
    int64_t rebuilds;   /* candidate-row rebuilds                                 */
    int64_t short_pairs;/* pair terms evaluated for F_0 (BOUNCE)                 */
    int64_t full_pairs; /* pair terms evaluated for the full gradient (BAOAB)    */
    double recip;       /* E_recip + E_self + E_exclusion of periodic Ewald (0)   */
} bounce_energies;

/* Launch parameters chosen by bounce_autotune. */
typedef struct bounce_tuning {
    int32_t tile_j;      /* atoms per j-block of the all-pairs tile kernel (0: not used)   */
    int32_t tile_blocks; /* its resident grid (CTAs of 256 threads)                        */
    double column_edge;  /* edge of the cluster columns in A (0: not used)                 */
    double pair_ms;      /* pair-sum kernel time of the chosen candidate, ms per launch    */
    int32_t candidates;  /* candidates timed                                               */
} bounce_tuning;

/* Fill *cfg with the defaults documented above. */
void bounce_config_default(bounce_config* cfg);

/* Create a context on cfg->device.  *out receives the context; the config
 * is copied.  Errors: INVALID_ARG (bad config), CUDA. */
int bounce_create(bounce_ctx** out, const bounce_config* cfg);

/* Topology (host arrays, copied).  type[n] in [0, BOUNCE_MAX_TYPES), mass[n]
 * (g/mol, > 0), charge[n] (e), molecule[n]: pairs within one molecule are
 * excluded from all pair terms and from the jump candidates.  bond_ij[2 nb],
 * bond_k_r0[2 nb]: E = k (r - r0)^2.  angle_ijk[3 na] (end, vertex, end),
 * angle_k_t0[2 na]: E = k (theta - theta0)^2, theta0 in rad.
 * Errors: INVALID_ARG, CUDA. */
int bounce_set_topology(bounce_ctx* ctx, int32_t n_atoms, const int32_t* type, const double* mass,
                        const double* charge, const int32_t* molecule, int32_t n_bonds, const int32_t* bond_ij,
                        const double* bond_k_r0, int32_t n_angles, const int32_t* angle_ijk,
                        const double* angle_k_t0);

/* Lennard-Jones table (host, copied): sigma[T*T], eps[T*T] per type pair,
 * E = 4 eps ((sigma/r)^12 - (sigma/r)^6); eps = 0 switches a pair off.
 * Computes the jump bounds L_ab = sup_r |chi W'_ab| (Sec. IV.A) for the
 * current topology and config.  Call after bounce_set_topology. */
int bounce_set_lj(bounce_ctx* ctx, int32_t n_types, const double* sigma, const double* eps);

/* Positions q[n,3] and velocities v[n,3] (A, A/fs); resets the step counter
 * to `step` (the Philox step index of the next step).  The candidate rows are
 * rebuilt at the next launch if this is the first state of the topology (or
 * of a replica layout) or if an atom lies more than skin/2 from its position
 * at the last row build -- the test a run applies every step; otherwise the
 * rows are kept.  Errors: INVALID_ARG, NONFINITE, STATE (no topology). */
int bounce_set_state(bounce_ctx* ctx, const double* q, const double* v, int64_t step, int32_t where, void* stream);

/* Copy the current state out (q, v may be NULL to skip). */
int bounce_get_state(bounce_ctx* ctx, double* q, double* v, int32_t where, void* stream);

/* Advance n_steps full steps of the integrator (BOUNCE_BAOAB,
 * BOUNCE_BOUNCE, BOUNCE_BOUNCE_RESPA, BOUNCE_BOUNCE_RESPA_EXT or
 * BOUNCE_BOUNCE_RESPA1); the returned state is after the last B half-kick.
 * With an SPME grid set, the reciprocal gradient is part of the full
 * gradient (BAOAB) or of F_0 (BOUNCE, Sec. V basic BOUNCE);
 * BOUNCE_BOUNCE_RESPA needs the grid; the RESPA integrators need a step
 * counter and n_steps that are multiples of respa_m (respa_m respa_m2 for
 * RESPA1) (else INVALID_ARG).  All
 * work stays on the device; the call does not synchronise `stream` except
 * to report row overflows, which it checks once at the end.
 * Errors: STATE, LIST_OVERFLOW (a row exceeded max_neighbors; the state is
 * then invalid), CUDA. */
int bounce_run(bounce_ctx* ctx, int64_t n_steps, int32_t integrator, void* stream);

/* Energies of the current state and the run counters (synchronises). */
int bounce_get_energies(bounce_ctx* ctx, bounce_energies* out, void* stream);

/* Zero the proposal / accept / tie / pair counters. */
int bounce_reset_counters(bounce_ctx* ctx, void* stream);

/* Jump bounds: L[T*T] (padded by 1e-6 relative) and row maxima Lstar[T]. */
int bounce_get_bounds(bounce_ctx* ctx, double* L, double* Lstar);

/* --- Component entry points (each runs the same kernels bounce_run uses). */

/* Gradient part (BOUNCE_GRAD_*) at the current positions into grad[n,3]. */
int bounce_compute_gradient(bounce_ctx* ctx, int32_t part, double* grad, int32_t where, void* stream);

/* One jump half-step J(delta/2) (Sec. IV.B, step J) on the current
 * velocities at the current positions, with the Philox counter of
 * (step, stream_id).  If M and n_acc are not NULL they receive, per atom,
 * the Poisson proposal count and the number of accepted reflections. */
int bounce_jump_half(bounce_ctx* ctx, int64_t step, int32_t stream_id, int32_t* M, int32_t* n_acc, int32_t where,
                     void* stream);

/* Candidate rows at the current positions (rebuilt first if stale):
 * counts[n] and rows[n * capacity] (ascending atom indices).  These are the
 * full rows (every atom of another molecule within r_c + skin) even where a
 * run's jump step reads rows restricted to the partners a jump can draw
 * (LJ alone on the jumps with one bound per type: see jump_coulomb); reading
 * them leaves the run's own rows and rebuild schedule unchanged. */
int bounce_get_rows(bounce_ctx* ctx, int32_t* counts, int32_t* rows, int32_t capacity);

/* Batch of independent replicas in one context (for example many small
 * droplets advanced together).  The topology holds all replicas back to back; replica r owns
 * atoms [atom_offsets[r], atom_offsets[r+1]) and draws every random number
 * with its own Philox key seeds[r] and its atoms' indices inside the
 * replica, so each replica follows exactly the trajectory it would follow
 * alone.  Pairs and jump candidates never cross replicas.  Replicas are open
 * droplets without a cutoff (every other-molecule atom of the replica);
 * max_neighbors must be at least the largest replica size - 1.  Every
 * bounce_run step then advances all replicas in the same kernel launches;
 * energies and counters are totals over the batch.  Call after
 * bounce_set_topology. */
int bounce_set_replicas(bounce_ctx* ctx, int32_t n_replicas, const int32_t* atom_offsets, const uint64_t* seeds);

/* Differentiable direct-space pair forces (force matching; the pair terms of
 * Sec. IV.A / V with trainable per-type parameters).  Parameters are host
 * tables: q_type[T] charges per atom type (replacing the topology charges in
 * these two calls), sigma[T*T] and eps[T*T] read from the upper triangle
 * (entry (a, b), a <= b, is the parameter of both orders).  Pairs: other
 * molecules with r^2 < r_c^2 (Coulomb or Ewald direct erfc, plus LJ); the
 * reciprocal and bonded parts are not included.
 *
 * bounce_pair_forward: with q (device [n,3]) non-NULL the positions are first
 * replaced and the rows rebuilt; forces (device [n,3]) receive
 * F_i = -dE_pair/dq_i and *energy (host, may be NULL) E_pair = sum_{i<j} W. */
int bounce_pair_forward(bounce_ctx* ctx, const double* q, int32_t n_types, const double* q_type, const double* sigma,
                        const double* eps, double* forces, double* energy, void* stream);

/* Backward of the last forward for a loss L(F, E): grad_forces (device
 * [n,3]) = dL/dF, grad_energy = dL/dE.  Receives grad_pos (device [n,3]) =
 * dL/dq (through the pair Hessian), and on the host grad_q_type[T],
 * grad_sigma[T*T], grad_eps[T*T] (entry (a, b) and (b, a) both hold the
 * derivative with respect to the shared table entry).  FP32 pair math, FP64
 * fixed-order reductions. */
int bounce_pair_backward(bounce_ctx* ctx, int32_t n_types, const double* q_type, const double* sigma,
                         const double* eps, const double* grad_forces, double grad_energy, double* grad_pos,
                         double* grad_q_type, double* grad_sigma, double* grad_eps, void* stream);

/* Observables (paper Sec. VI). */

/* Counts of unordered pairs (different molecules) of the type pair
 * {type_a, type_b} by distance, n_bins bins of width r_max / n_bins over
 * [0, r_max) (bin k: (k w)^2 <= r^2 < ((k+1) w)^2 in FP64); hist[n_bins]
 * (host) receives the counts.  Needs r_max <= r_c when a cutoff is set.
 * Synchronises `stream`. */
int bounce_pair_histogram(bounce_ctx* ctx, int32_t type_a, int32_t type_b, double r_max, int32_t n_bins,
                          int64_t* hist, void* stream);

/* Take the current (unwrapped) positions as the reference of bounce_msd. */
int bounce_set_msd_reference(bounce_ctx* ctx, void* stream);

/* Mean over atoms of `type` of |q_i - q_i(ref)|^2 (A^2), FP64, into *out.
 * Synchronises `stream`. */
int bounce_msd(bounce_ctx* ctx, int32_t type, double* out, void* stream);

/* Profiling: advance n_steps exactly as bounce_run does, but with direct
 * launches (no graph) and CUDA events around every launch of the fused step
 * kernel; *kernel_ms receives the summed step-kernel time and *launches
 * the number of step-kernel launches.  Synchronises `stream`. */
int bounce_profile_steps(bounce_ctx* ctx, int64_t n_steps, int32_t integrator, void* stream, double* kernel_ms,
                         int64_t* launches);

/* Autotuner: times the pair-sum kernel of `integrator` on the current state
 * for each candidate launch shape and keeps the fastest for later runs.
 * Systems without a cutoff (droplets, replica batches): the j-block length
 * of the all-pairs tiles (32, 64, 128, 256 atoms) and the resident grid
 * (2, 4, 8 CTAs per SM); systems with a cutoff: the edge of the cluster
 * columns (0.8 to 1.25 times (8 / density)^(1/3)).  The results of a run do
 * not depend on the choice except through the order of FP32 partial sums.
 * Captured graphs are dropped.  *out receives the choice.  Synchronises
 * `stream`.  Errors: STATE (no state), CUDA. */
int bounce_autotune(bounce_ctx* ctx, int32_t integrator, void* stream, bounce_tuning* out);

/* Profiling breakdown: advance n_steps exactly as bounce_run does, but with
 * direct launches (no graph) and CUDA events around each group of launches
 * of every step boundary.  ms[5] receives the summed device time of
 * (0) the pair-sum kernel, (1) the step kernel, (2) the candidate-row
 * rebuild launches, (3) the cluster-list rebuild launches, (4) the SPME
 * launches; groups[5] (may be NULL) the number of boundaries timed for each
 * (a gated rebuild that finds nothing to do still counts).  Synchronises
 * `stream`.  Errors: as bounce_run. */
int bounce_profile_breakdown(bounce_ctx* ctx, int64_t n_steps, int32_t integrator, void* stream, double* ms,
                             int64_t* groups);

/* Number of kernel launches a bounce_run of n_steps of `integrator` would
 * issue from the current state (launch accounting: gated row-rebuild
 * launches, step kernels, SPME launches, step-counter updates). */
int64_t bounce_run_launch_count(const bounce_ctx* ctx, int64_t n_steps, int32_t integrator);

/* Allocation-free pair energies.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code that
 * lives inside an allocator owning the whole device pool (a foreign
 * cudaMalloc would escape its accounting), hosts that forbid allocation after
 * start-up (embedded or real-time loops, where cudaMalloc may block and
 * synchronise the device), and plug-ins handed device buffers but no right to
 * allocate.
 * It returns out[0] = sum_{i<j} k q_i q_j / r (or erfc(beta r)/r with
 * ewald_beta > 0) and out[1] = sum_{i<j} 4 eps ((sigma/r)^12 - (sigma/r)^6)
 * over all pairs of different molecules with r < r_cut (r_cut <= 0 or inf:
 * no cutoff; box = NULL: open boundaries, else 3 host doubles for a periodic
 * box, which needs a finite r_cut <= min(box)/2 so that the minimum image is
 * the pair sum), the same totals as bounce_get_energies' coulomb and lj.
 * Inputs are caller-owned DEVICE arrays of the current device, contiguous:
 * q[n,3] double, charge[n] double, type[n] int32 with 0 <= type < n_types,
 * molecule[n] int32; sigma and eps are host T*T tables (T = n_types); out is
 * a DEVICE array of 2 doubles written on `stream`.  A type outside
 * [0, n_types) is not read from the tables: both totals are then NaN.
 * The call allocates nothing: its scratch is a static device array of
 * BOUNCE_NOALLOC_MAX_ATOMS atoms plus a status word (786,688 bytes) that
 * every GPU loading this library holds until exit.  n > BOUNCE_NOALLOC_MAX_ATOMS
 * returns BOUNCE_ERR_INVALID_ARG.  The first call on a device looks up the
 * scratch address on that device (make it before any stream capture).
 * Calls share the scratch: calls whose GPU work overlaps race.  An error
 * already pending on the calling thread (from earlier, unrelated work) is
 * left in place and the call returns BOUNCE_ERR_CUDA without launching. */
int bounce_pair_energy_noalloc(int32_t n, const double* q, const double* charge, const int32_t* type,
                               const int32_t* molecule, int32_t n_types, const double* sigma, const double* eps,
                               double r_cut, double ewald_beta, const double* box, double* out, void* stream);

/* Message of the last error on ctx (never NULL). */
const char* bounce_last_error(const bounce_ctx* ctx);

/* Free all device and host memory of ctx. */
void bounce_destroy(bounce_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* BOUNCE_H */
