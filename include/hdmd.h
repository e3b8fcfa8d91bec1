/*
 * hdmd.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * d-dimensional soft-sphere molecular dynamics of Hoy & Interiano-Alberto,
 * "Efficient d-dimensional molecular dynamics simulations for studies of the
 * glass-jamming transition" (arXiv:2112.12271).
 *
 * What one system holds: N spheres in a periodic hypercube of side L centred
 * at the origin, 2 <= d <= 10 (Sec. II: all routines work in any d), with
 * per-sphere diameters sigma_i, masses m_i, positions, velocities, image
 * counts, the linked-subcell structure (Sec. II.C, Eqs. (7)-(9)) and a full
 * Verlet list with skin s.  All of it lives in GPU memory owned by the
 * library.  The compute steps (binning, list build, forces, integration,
 * FIRE, SWAP) run as CUDA kernels on the stream given at creation.
 *
 * Conventions for every call:
 *   - returns an hdmd_status; never aborts, throws or exits;
 *   - host arrays are owned by the caller and copied (pinned memory makes
 *     the copies asynchronous-capable, pageable memory also works);
 *   - positions and velocities cross the ABI row-major, x[i*d + k], in the
 *     caller's atom order; the library may reorder atoms internally but
 *     every output is returned in the caller's order;
 *   - calls on one system are not thread-safe; distinct systems are
 *     independent;
 *   - on failure hdmd_last_error() describes the cause.
 */
#ifndef HDMD_H
#define HDMD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hdmd_system hdmd_system; /* opaque, library-owned */

typedef enum {
    HDMD_OK = 0,
    HDMD_E_INVALID = 1,        /* bad argument (sizes, box too small, NaN input) */
    HDMD_E_NOMEM = 2,          /* device allocation failed */
    HDMD_E_NBR_OVERFLOW = 3,   /* list capacity exceeded and could not be grown */
    HDMD_E_LOST_ATOM = 4,      /* non-finite coordinates or a displacement beyond the skin */
    HDMD_E_NOT_CONVERGED = 5,  /* FIRE stopped at max_iter or on the P<=0 limit */
    HDMD_E_CUDA = 6,           /* a CUDA runtime call failed */
    HDMD_E_TIMEOUT = 7,        /* a bounded device-side wait ran out */
    HDMD_E_UNSUPPORTED_D = 8   /* d outside 2..10 */
} hdmd_status;

typedef enum { HDMD_FP64 = 0, HDMD_MIXED = 1 } hdmd_precision;

/* Pair law, with the Lorentz mixing rule sigma_ij = (sigma_i + sigma_j)/2
 * (Sec. II.A; the paper states the radial law is a user choice).
 *   kind 0: harmonic soft spheres
 *     U(r) = (eps_ij/2) (1 - r/sigma_ij)^2 for r < sigma_ij, 0 beyond;
 *   kind 1: the paper's truncated and shifted Morse law, Eq. (1),
 *     U(r) = eps_ij [exp(-2a(r - sigma_ij)) - 2 exp(-a(r - sigma_ij)) + 1]
 *     for r < sigma_ij, 0 beyond (a > 0: stiffness; the paper uses 30).
 *   kind 2: the Mie law of Sec. II.A truncated at its minimum sigma_ij (the
 *     paper's default cut) and shifted to be continuous there,
 *     U(r) = eps_ij [(sigma_ij/r)^(2n) - 2 (sigma_ij/r)^n + 1] for
 *     r < sigma_ij, 0 beyond (n = n_mie in 1..24; n = 6 is the WCA form).
 * eps_scale 0: eps_ij = eps for every pair; 1: each atom has the prefactor
 * eps_i = eps sigma_i^d (prefactors scale with particle volume, Sec. II.A)
 * and eps_ij = sqrt(eps_i eps_j) (the mixing rule of Sec. II.A).
 * skin: the Verlet-list skin s of Sec. II.C (list radius sigma_ij + s).
 * Other kinds, a <= 0 for kind 1, n_mie outside 1..24 for kind 2, or
 * eps_scale outside {0, 1} are rejected
 * with HDMD_E_INVALID.  The batched engine and the allocation-free force
 * call use kind 0 with one eps. */
typedef struct {
    int kind;
    double eps;
    double skin;
    double a;
    int eps_scale;
    int n_mie;
} hdmd_potential;

/* Thermodynamic summary (Sec. II.E): pair energy E = sum_{i<j} U_ij, virial
 * W = sum_{i<j} r_ij . f_ij, kinetic K = sum m v^2 / 2, T = 2K/(d(N-1)),
 * P = (2K + W)/(d V).  steps/rebuilds count what the call did. */
typedef struct {
    double E_pair, virial, K, T, P;
    int64_t steps, rebuilds;
} hdmd_thermo;

/* FIRE 2.0 settings (Sec. II.B; constants of the published FIRE 2.0).
 * f_tol: stop when max_i |F_i| < f_tol.  polish_tol: in HDMD_MIXED systems
 * the iteration runs with FP32 pair forces until max_i |F_i| < polish_tol
 * times the law's stiffness factor (1 harmonic, 2 (a max sigma)^2 Morse), or
 * until n_neg_max P <= 0 steps in a row show that FP32 rounding stalls it,
 * then continues with FP64 pair forces (0 disables the switch).
 * The paper's own criteria and cap (Sec. II.B, Table II; each off when 0):
 * e_thres stops when the average pair energy E_pair/N < e_thres (the
 * paper's pushoff uses e_thres = eps); f_thres stops when the fractional
 * drop |(E_{i+1} - E_i)/E_i| (Eq. (6)) stays below it for ten consecutive
 * iterations; dx_max > 0 caps each atom's move per iteration (the step
 * dt v_i and the back-off (dt/2) v_i) at length dx_max (system path only;
 * the batched engine rejects it). */
typedef struct {
    double dt0, dt_max, dt_min, f_inc, f_dec, alpha0, f_alpha, f_tol, polish_tol;
    int64_t n_delay, n_neg_max, max_iter;
    int initial_delay;
    double e_thres, f_thres, dx_max;
} hdmd_fire_params;

typedef struct {
    int64_t iterations;        /* FIRE iterations run */
    int64_t polish_iterations; /* of which with FP64 pair forces */
    int64_t rebuilds;          /* Verlet-list builds during the call */
    double E_pair;             /* final pair energy */
    double fmax;               /* final max_i |F_i| */
    int converged;             /* 1 if fmax < f_tol */
} hdmd_fire_result;

typedef struct {
    int d;
    int64_t N;
    double L;
    int n_cell;                /* subcells per axis, Eq. (7) */
    int64_t n_cells;           /* n_cell^d */
    int list_capacity;         /* entries per atom currently allocated */
    int lanes_per_atom;        /* threads cooperating on one atom's list */
    int max_list_length;       /* longest list at the last build */
    int64_t total_list_entries;/* sum of list lengths at the last build */
    int precision;             /* hdmd_precision */
    int graphs;                /* 1 if CUDA graphs with conditional nodes are used */
    int64_t device_bytes;      /* device memory held by the system */
    int resident;              /* blocks of the resident MD kernel that md_steps
                                  would launch now (0: one kernel per step) */
} hdmd_info;

/* Device bytes that create_system would allocate for these arguments (the
 * lists at their initial capacity; they grow on overflow).  Same argument
 * checks as create_system; no device work.  Lets a scheduler admit a job by
 * free device memory before it creates the system.  *bytes receives it. */
hdmd_status system_footprint(int d, int64_t N, double L, const double *diameters,
                             const hdmd_potential *pot, hdmd_precision prec, int64_t *bytes);

/* Create a system: d in 2..10 (else HDMD_E_UNSUPPORTED_D), N >= 2 atoms,
 * box side L, diameters[N] (host, > 0 and finite, copied).  Requires
 * L > 2 max sigma, so that only one periodic image of a pair can interact.
 * The subcells per axis are n_cell = floor(L/(max sigma + skin)) (Eq. (7));
 * when that is 1 the lists are built over all pairs.  prec selects FP64 or mixed
 * (FP32 pair arithmetic; FP64 positions, velocities and reductions).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every
 * kernel of this system runs.  Positions start at the origin: call
 * set_state before anything else.  *out receives the handle. */
hdmd_status create_system(int d, int64_t N, double L, const double *diameters,
                          const hdmd_potential *pot, hdmd_precision prec,
                          void *cuda_stream, hdmd_system **out);

/* Load positions x[N*d] (host, row-major, any real values: wrapped into the
 * box), velocities v[N*d] (nullable: zero) and masses[N] (nullable: all 1,
 * positive).  Resets image counts to 0 and forces a list rebuild. */
hdmd_status set_state(hdmd_system *sys, const double *x, const double *v,
                      const double *masses);

/* Change the diameters (host [N], copied); forces a rebuild. */
hdmd_status set_diameters(hdmd_system *sys, const double *diameters);

/* Read back positions wrapped into [-L/2, L/2), velocities, image counts
 * img[N*d] (x + img L is the unwrapped position), forces f[N*d] at the
 * current positions and diameters[N].  Every output is nullable.
 * Synchronises the stream. */
hdmd_status get_state(hdmd_system *sys, double *x, double *v, int32_t *img,
                      double *f, double *diameters);

/* Build the cell structure and Verlet lists (Sec. II.C).  force != 0
 * rebuilds unconditionally; force == 0 rebuilds only if the displacement
 * trigger fires: 2 max_i |x_i - x_i(last build)| > skin.  *rebuilt (nullable)
 * receives 1 if a build happened. */
hdmd_status build_neighbors(hdmd_system *sys, int force, int *rebuilt);

/* Test hook: the current full lists in caller order.  counts[N] receives
 * each list length; idx (nullable; room for sum(counts) entries) receives
 * the lists back to back, each sorted ascending.  *total (nullable)
 * receives sum(counts). */
hdmd_status get_neighbors(hdmd_system *sys, int32_t *counts, int32_t *idx,
                          int64_t *total);

/* Pair forces, energy and virial at the current positions (Sec. II.B
 * getforce), rebuilding the lists first if the trigger fires.  energy and
 * virial (nullable) receive E_pair and W; forces are kept on the device
 * (get_state reads them). */
hdmd_status compute_forces(hdmd_system *sys, double *energy, double *virial);

/* nsteps of kick-drift-kick velocity Verlet (Sec. II.B) with time step dt,
 * in NVE or, after set_thermostat, NVT; the displacement trigger is checked
 * after every drift on the device and the lists rebuilt there when it
 * fires.  last (nullable) receives the thermodynamic state after the final
 * step.  On list overflow the call restores its starting state, grows the
 * lists and runs again. */
hdmd_status md_steps(hdmd_system *sys, int64_t nsteps, double dt, hdmd_thermo *last);

/* Berendsen barostat (Berendsen et al. 1984; the NPT control of Sec. II.E).
 * With tau_P > 0, md_steps runs in pieces of n_baro steps; after each full
 * piece (counted across calls) the pressure P = (2K + W)/(d L^d) of its end
 * state gives mu = [1 - beta (n_baro dt / tau_P)(P_target - P)]^(1/d), every
 * position and the box side are multiplied by mu (box centred at the
 * origin), the subcell grid of Eq. (7) is set up again for the new box and
 * the lists are rebuilt (as the paper's Berendsen() does when n_cell
 * changes).  beta: compressibility (> 0); n_baro >= 1.  tau_P <= 0 turns it
 * off.  md_steps fails with HDMD_E_INVALID if a rescaling would leave the
 * box below twice the largest diameter; hdmd_info.n_cell and get_box report
 * the current box. */
hdmd_status set_barostat(hdmd_system *sys, double P_target, double tau_P, double beta,
                         int64_t n_baro);

/* List rebuild rule.  rule 0 (default): rebuild as soon as 2 max_i |x_i -
 * x_i(build)| > s, checked after every drift, which keeps the forces exact.
 * rule 1: the paper's rule (Sec. II.C), checked after every n_bet-th MD
 * step (counted from this call on): rebuild when at least 0.1 % of the
 * atoms have moved by s/2 or any atom by s; it can miss a pair closing from
 * both sides, so forces may deviate from the exact ones.  FIRE keeps rule 0. */
hdmd_status set_rebuild_rule(hdmd_system *sys, int rule, int n_bet);

/* List radius: global 0 (default) keeps pair (i, j) in the lists when
 * r < sigma_ij + s; global 1 uses the paper's single radius
 * r_c^max = sigma_max + s (Sec. II.C) for every pair (longer lists, same
 * forces).  The lists are rebuilt at once. */
hdmd_status set_list_radius(hdmd_system *sys, int global);

/* Current box side (it changes under the barostat). */
hdmd_status get_box(hdmd_system *sys, double *L);

/* Observables of Sec. II.E against a reference configuration (the paper's
 * r_i(0), taken at step n_msdstart):
 *   msd = <|dr|^2>, mqd = <|dr|^4> over the N atoms, dr = unwrapped
 *   displacement since the reference;
 *   alpha2 = d mqd / ((d + 2) msd^2) - 1, the non-Gaussian parameter (Eq. (14));
 *   f_ov = fraction of atoms with |dr| < a, the overlap function (Eq. (15),
 *   whose threshold is 0.1 d in units of the typical diameter);
 *   Z = mean number of neighbours closer than sigma_ij (coordination number). */
typedef struct {
    double msd, mqd, alpha2, f_ov, Z;
} hdmd_observables;

/* Store the reference configuration: x_ref[N*d] (host, row-major, caller
 * order, unwrapped) or, when NULL, the current unwrapped positions. */
hdmd_status set_reference(hdmd_system *sys, const double *x_ref);

/* Observables at the current positions against the stored reference
 * (HDMD_E_INVALID without one).  a_ov: overlap threshold (<= 0: 0.1 d).
 * gs (nullable, host [nbins]) receives the self part of the van Hove
 * function (Eq. (16)) as a histogram: gs[b] = (atoms with b w <= |dr| <
 * (b + 1) w) / (N w), w = r_max / nbins; nbins in 0..65536 (0: none),
 * r_max > 0 when nbins > 0. */
hdmd_status observables(hdmd_system *sys, double a_ov, int nbins, double r_max,
                        hdmd_observables *out, double *gs);

/* Berendsen thermostat (Berendsen et al. 1984; the NVT control of
 * Sec. II.E, which the paper applies inside the second kick of each step,
 * Sec. II.B).  With tau > 0 every later md_steps ends each step's second
 * kick with v *= lambda, lambda = sqrt(1 + (dt/tau)(T_target/T - 1)), T the
 * kinetic temperature 2K/(d(N-1)) at the end of the previous step (at the
 * start of the call for its first step; lambda = 1 when T = 0).  tau <= 0
 * returns to NVE.  T_target must be >= 0 and finite (HDMD_E_INVALID). */
hdmd_status set_thermostat(hdmd_system *sys, double T_target, double tau);

/* FIRE 2.0 minimisation (Sec. II.B names the method; the steps are those
 * of the published FIRE 2.0 algorithm, Guenole et al. 2020: on P = F.v <= 0
 * past the initial delay dt *= f_dec only while f_dec dt >= dt_min, and
 * alpha = alpha0; x -= dt v/2, v = 0; then in every iteration v += dt F/m,
 * v = (1 - alpha) v + alpha |v| F/|F| over all atoms, x += dt v).
 * params NULL takes the defaults
 * (dt0 0.005, dt_max 0.05, dt_min 1e-4, f_inc 1.1, f_dec 0.5, alpha0 0.25,
 * f_alpha 0.99, f_tol 1e-10, polish_tol 1e-6, n_delay 20, n_neg_max 2000,
 * max_iter 10^6, initial_delay 1).  Velocities are zeroed on entry and the
 * minimised positions replace the state.  Returns HDMD_E_NOT_CONVERGED,
 * with *res filled, when it stops without reaching f_tol. */
hdmd_status fire_minimize(hdmd_system *sys, const hdmd_fire_params *params,
                          hdmd_fire_result *res);

/* SWAP Monte Carlo (Sec. II.D): nsweeps passes of round(p N) candidate
 * exchanges each, at temperature T.  With pairs == NULL the candidates and
 * the Metropolis uniforms come from Philox4x32-10 keyed by seed (pass s,
 * pair k at counter (k, s, 0x53574150, 0)); otherwise pairs[2*npairs]
 * (host, caller order, i != j) and uniforms[npairs] in [0,1) give one pass
 * explicitly and p, seed and nsweeps are ignored.  The outcome equals
 * serial execution of the candidates in order.  *accepted (nullable)
 * receives the number of accepted exchanges; accepted_flags (nullable,
 * host, npairs bytes) receives each decision of an explicit pass. */
hdmd_status swap_sweep(hdmd_system *sys, int nsweeps, double T, double p,
                       uint64_t seed, const int32_t *pairs, const double *uniforms,
                       int64_t npairs, int64_t *accepted, uint8_t *accepted_flags);

/* Introspection and tuning. lanes_per_atom in {1,2,4,8,16,32} (0 keeps the
 * current value); use_graphs 0/1 (-1 keeps).  Takes effect at the next
 * list build, which this call forces. */
hdmd_status get_info(hdmd_system *sys, hdmd_info *info);
hdmd_status set_tuning(hdmd_system *sys, int lanes_per_atom, int use_graphs);

/* Resident MD (on = 1, the default): in mixed precision with the exact
 * rebuild rule, md_steps runs the steps between list builds (Sec. II.C) in
 * one cooperative launch whose blocks keep their atoms' state and lists in
 * shared memory and exchange positions through L2 each step; it applies
 * when the per-atom state fits in shared memory (about 10^5 atoms at d = 6
 * on GB300).  The trajectory is the same, bit for bit in NVE, as with
 * on = 0 (one kernel launch per step).  A block that waits too long for the
 * others makes md_steps return HDMD_E_TIMEOUT. */
hdmd_status set_resident(hdmd_system *sys, int on);

/* Benchmark support, not part of the method: average device time in
 * milliseconds of single kernels on the current state, each launch timed
 * alone with a CUDA event pair on the system's stream and averaged over reps
 * launches.  ms_out (host, 4 doubles)[0]: the fused MD kernel (pair forces
 * over the list, both half kicks, drift, trigger reduction) with time step
 * dt; [1]: one full list build (wrap, binning, counting sort, reorder,
 * Verlet lists); [2]: the force-only kernel; [3]: the resident MD kernel,
 * one launch of up to 20 reps steps divided by the steps it ran (0 where
 * md_steps would not use it).  The state (positions, velocities, lists) is
 * restored before returning. */
hdmd_status profile_kernels(hdmd_system *sys, int reps, double dt, double *ms_out);

/* Forces, pair energy and virial of N harmonic spheres, for callers that
 * cannot allocate GPU memory when they need them: plug-ins inside a host
 * framework whose memory pool owns the device (a cudaMalloc of their own
 * would bypass, or fail under, that pool's budget), and loops that forbid
 * allocation after start-up (an allocation can block on the whole device
 * and its time is unbounded).  The paper has no counterpart of this call; it
 * is the FP64 force kernel with all pairs in place of the Verlet list, so it
 * needs no system handle, no list and no cell arrays.
 * Cost: all N^2 pairs in FP64, O(N^2 d) work, which the narrow FP64 pipe of
 * this GPU makes the bound; it suits small and mid-size systems, not the
 * largest N it accepts.  Measured on one GB300: 12 ms per call at d = 3,
 * N = 16384; 22 ms at d = 6, N = 16384; 0.32 s at d = 6, N = 65536 (so
 * about 80 s at the 524288-atom limit).
 * Arguments: d in 2..10; N atoms, 2 to 524288; box side L, which must be at
 * least twice the largest diameter (not checked: the kernel evaluates the
 * nearest image of each pair, which is then the only image that can
 * overlap; in a smaller box a pair can also overlap through a farther image,
 * which is left out); device pointers x_dev
 * [N*d] row-major positions, sigma_dev [N] diameters, F_dev [N*d] forces out,
 * ew_dev [2] out (pair energy, virial); eps as in hdmd_potential; cuda_stream
 * a cudaStream_t (NULL = legacy default stream).  The call is asynchronous:
 * the outputs are ready when the stream reaches it.
 * Memory: it allocates nothing.  Its only scratch is a file-scope device
 * array of 65,792 bytes that every GPU loading the library holds until the
 * process exits.  The first call on a device looks up that array's device
 * address (once per device, with the device current).  All calls share the
 * array and it keeps the last call's contents (the call clears what must
 * start at zero), so calls that overlap on the GPU, on any streams, race:
 * serialise them.
 * Errors: HDMD_E_UNSUPPORTED_D, HDMD_E_INVALID (N out of range, NULL
 * buffer, bad L or eps), HDMD_E_CUDA; hdmd_noalloc_last_error() gives the
 * reason. */
hdmd_status compute_forces_noalloc(int d, int64_t N, double L, const double *x_dev,
                                   const double *sigma_dev, double eps, double *F_dev,
                                   double *ew_dev, void *cuda_stream);
const char *hdmd_noalloc_last_error(void);

/* ------------------------------------------------------------------------
 * Batched jobs: many independent systems of uneven N and d advanced by one
 * persistent kernel per dimension (one thread block per job at a time), for
 * throughput on many small systems and for the serving loop.  Each job runs
 * the same method as a single system (lists over the 3^d subcells, pair
 * forces, FIRE 2.0 or velocity Verlet) with unit masses.
 * ---------------------------------------------------------------------- */
typedef struct hdmd_batch hdmd_batch;

typedef struct {
    int kind;             /* 0: MD (nsteps of velocity Verlet, step dt), 1: FIRE */
    int d;                /* 2..10 */
    int64_t N;
    double L, eps, skin;
    double dt;            /* MD */
    int64_t nsteps;       /* MD */
    int list_capacity;    /* 0: estimated from the density */
    hdmd_fire_params fire;/* FIRE; dt0 <= 0 takes the defaults of fire_minimize */
} hdmd_job_spec;

typedef struct {
    int status;           /* 0 running, 1 done, 2 FIRE stopped unconverged, 3 error */
    int kind;
    int64_t iterations;   /* FIRE iterations or MD steps done */
    int64_t rebuilds;
    double E_pair, virial, K, fmax;
    int converged;        /* FIRE: max_i |F_i| < f_tol */
    int error;            /* 1: list overflow (re-admit with a larger list_capacity), 2: lost atom */
} hdmd_job_result;

/* A batch with a device pool of pool_bytes (cudaMalloc once) and room for
 * max_jobs jobs; prec as for create_system; kernels run on cuda_stream. */
hdmd_status batch_create(int64_t pool_bytes, int max_jobs, hdmd_precision prec,
                         void *cuda_stream, hdmd_batch **out);
/* Admit one job: diameters[N], positions x[N*d] (row-major, host), velocities
 * v[N*d] (nullable).  Its memory is carved out of the pool; HDMD_E_NOMEM when
 * the pool (or the job table) has no room now: remove finished jobs first.
 * *job_id receives the job's slot. */
hdmd_status batch_add(hdmd_batch *b, const hdmd_job_spec *spec, const double *diameters,
                      const double *x, const double *v, int *job_id);
/* One launch over every running job: each advances by at most budget FIRE
 * iterations or MD steps (0: until it finishes).  *n_unfinished (nullable)
 * receives the number still running.  Synchronises the stream. */
hdmd_status batch_run(hdmd_batch *b, int64_t budget, int *n_unfinished);
/* Result of a job (finished or not); x (nullable, host [N*d]) receives its
 * positions wrapped into the box, in the caller's atom order. */
hdmd_status batch_result(hdmd_batch *b, int job_id, hdmd_job_result *res, double *x);
/* Return a job's memory to the pool and free its slot. */
hdmd_status batch_remove(hdmd_batch *b, int job_id);
/* Free pool bytes, live jobs, lanes per atom by dimension (int[11]); nullable. */
hdmd_status batch_info(hdmd_batch *b, int64_t *free_bytes, int *live_jobs, int *lanes_by_d);
/* Autotuner of the block shape per dimension: times the force evaluation of
 * each dimension's median job with 1..16 lanes per atom (reps evaluations,
 * CUDA events) and keeps the fastest for that dimension. */
hdmd_status batch_autotune(hdmd_batch *b, int reps);
/* Set the lanes per atom (power of two, 1..16) of a dimension by hand. */
hdmd_status batch_set_lanes(hdmd_batch *b, int d, int lanes);
hdmd_status batch_destroy(hdmd_batch *b);
const char *hdmd_batch_last_error(const hdmd_batch *b);

/* Free everything the system holds.  NULL is accepted. */
hdmd_status destroy_system(hdmd_system *sys);

/* Description of the last failure on sys, or of the last failure of this
 * thread when sys is NULL.  Never NULL; valid until the next call. */
const char *hdmd_last_error(const hdmd_system *sys);

#ifdef __cplusplus
}
#endif
#endif /* HDMD_H */
