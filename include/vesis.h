/*
 * vesis.h - C ABI of the GB300 (sm_103a) VESIS hot path.
 *
 * Variational explicit-solute implicit-solvent relaxation of Liu, Zhang,
 * Cheng and Li (arXiv 2208.05524): the free energy G[Gamma, R] of
 * Eq. (freeenergyfn) is minimised by alternating the binary level-set
 * method (Sec. 3.1) at fixed atoms and adaptive-mobility gradient descent
 * of the atoms (Sec. 3.2) at a fixed interface (Sec. 3.3, Steps 1-5).
 *
 * Units: Angstrom, k_B T, elementary charge.  Host arrays are FP64.
 *
 * Grid: nx * ny * nz cells of side h; cell (i,j,k) has its centre at
 * origin + (i + 1/2, j + 1/2, k + 1/2) h and linear index
 * (i * ny + j) * nz + k (z fastest).  The box is the union of the cells.
 * Labels chi are uint8, 1 = solute (phi = -1 in the paper), 0 = solvent;
 * cells outside the box count as solvent.
 *
 * Device arrays (suffix _dev) are raw device pointers on the device that
 * was current when the system was created (for example the data_ptr() of
 * contiguous CUDA tensors).  The caller owns every array it passes; the
 * library owns only its internal scratch, released by vesis_destroy.
 * Work is enqueued on the stream given to vesis_init_system; calls that
 * return host values synchronise that stream before returning.
 *
 * Errors: every call returns a vesis_status.  Negative values are errors
 * (nothing is guaranteed about outputs), positive values are warnings
 * (outputs valid).  vesis_last_error() gives a thread-local message for
 * the last failing call on the calling thread.  No call aborts the process.
 */
#ifndef VESIS_H
#define VESIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VESIS_OK = 0,
    VESIS_E_ARG = -1,          /* invalid argument or size */
    VESIS_E_CUDA = -2,         /* CUDA runtime error */
    VESIS_E_NAN = -3,          /* non-finite energy or gradient */
    VESIS_E_OUT_OF_BOX = -4,   /* an atom left the box */
    VESIS_E_ALLOC = -5,        /* device allocation failed */
    VESIS_W_MAX_ROUNDS = 1,    /* flip rounds hit their cap */
    VESIS_W_NOT_CONVERGED = 2  /* relaxation hit k_max or the retry cap */
} vesis_status;

/* Model and discretisation parameters.  vesis_default_params() fills the
 * paper's Table 1 (T = 298 K, rho_w = 0.0333 A^-3, gamma0 = 0.174 kBT/A^2,
 * eps_m = 1, eps_w = 80) and the discretisation described below. */
typedef struct {
    double gamma0;       /* surface tension, kBT/A^2 (Eq. G_VISM) */
    double rho_w;        /* solvent number density, A^-3 */
    double eps_m;        /* solute relative permittivity */
    double eps_w;        /* solvent relative permittivity */
    double temperature;  /* K; fixes k_B T and the Bjerrum length */
    double eps_ss;       /* permittivity of solute-solute Coulomb (Eq. Gss);
                            default eps_m */
    int nx, ny, nz;      /* grid cells per axis, each 1..4096 */
    double h;            /* grid spacing, A */
    double origin[3];    /* lower box corner, A */
    double gauss_sigma;  /* surface kernel width, A; <= 0 means 2 h */
    int trunc_r;         /* kernel half-width in cells, 1..8 (default 6) */
    double r_min;        /* distance clamp of every pair term, A (0.2) */
    int far_field;       /* 1: include the integral outside the box */
    int far_nuv;         /* far-field Gauss points per face axis (16) */
    int far_nt;          /* far-field Gauss points along rays (8) */
    int kernel;          /* surface kernel: 0 = separable truncated Gaussian
                            (gauss_sigma, trunc_r); 1 = the paper's
                            K = sin^2(pi |x| / delta) on |x| <= delta =
                            sin2_lambda sqrt(h) (Sec. 3.1), integer weights
                            round(2^16 K); delta / h must give 1..8 cells */
    double sin2_lambda;  /* lambda of delta = lambda sqrt(h) (default 2) */
} vesis_params;

/* Algorithm constants of Step 1 (defaults: k_max = 3000, N*_cnt = 5,
 * window 100, M = 1, alpha = 1/sqrt(2), delta G* = 5% of |G_old|,
 * Tol1 = 1e-4, Tol2 = 1e-5) and the caps this implementation adds. */
typedef struct {
    int max_outer;        /* k_max */
    int ncnt_star;        /* N*_cnt */
    int window;           /* steps the energy test must hold (Step 5) */
    double M0;            /* initial M */
    double alpha;         /* shrink factor of M */
    double dgstar_frac;   /* delta G* = dgstar_frac * |G_old| */
    double tol_grad;      /* Tol1: max |dG/dr| (Step 3.2) */
    double tol_energy;    /* Tol2: abs or rel energy change (Step 5) */
    int max_flip_rounds;  /* cap on flip rounds per interface relaxation */
    int max_gd_retries;   /* cap on consecutive shrinks of M (Step 3.4) */
    int resume;           /* 0: start afresh (k = 0, M = M0, N_cnt = 0);
                             1: continue from the system's relaxation state
                             (vesis_get_state / vesis_set_state), with
                             max_outer the cap on the total k */
} vesis_relax_opts;

/* Where a relaxation stands between two outer iterations (Sec. 3.3): with
 * the labels and positions it ended at, enough to continue it exactly as
 * if it had not stopped.  Plain data: save it beside chi and xyz to
 * checkpoint a relaxation, load it into any system of the same solute to
 * resume. */
typedef struct {
    int k;            /* accepted outer iterations so far */
    int ncnt;         /* N_cnt, accepted steps since M last shrank (Step 3.4) */
    int stable;       /* consecutive steps the energy test of Step 5 has held */
    int valid;        /* 1 once a relaxation has ended normally or by a cap */
    double M;         /* the mobility factor M (Eq. adjustmml) */
    double G_prev;    /* total G at the last accepted iterate (Steps 4-5) */
} vesis_relax_state;

/* Per-run report of vesis_relax. */
typedef struct {
    int status;            /* vesis_status of the run */
    int iterations;        /* accepted outer iterations k */
    int stop_reason;       /* 0 gradient test, 1 energy test, 2 k_max,
                              3 retry cap */
    long long flip_rounds; /* flip rounds over all outer iterations */
    long long flips;       /* flipped cells over all outer iterations */
    long long gd_trials;   /* trial positions evaluated (accepts+rejects) */
    long long pair_evals;  /* atom-point pair evaluations issued */
    double G;              /* final total free energy, kBT */
    double terms[6];       /* surface, vdW, CFA, far field, solute-solute,
                              total at the final state */
    double M;              /* final mobility factor */
    double max_grad;       /* max |dG/dr| at the last gradient evaluation */
    int records;           /* per-iteration records written (vesis_set_history) */
} vesis_relax_stats;

/* One accepted outer iteration of vesis_relax (Sec. 3.3, Steps 2-4). */
typedef struct {
    int k;              /* the iterate's number (1, 2, ...; continues on resume) */
    int rounds;         /* flip rounds of the iteration's interface relaxation */
    long long flips;    /* cells flipped by it */
    int trials;         /* trial positions evaluated: rejections + the accept */
    int ncnt;           /* N_cnt after the accept */
    double G;           /* total G at the accepted iterate (Gamma^{k}, R^{k}) */
    double G_old;       /* total G at (Gamma^{k}, R^{k-1}), before the step */
    double M;           /* mobility factor after the step */
    double max_grad;    /* max |dG/dr| that set the step (Eq. adjustmml) */
} vesis_iter_record;

typedef struct vesis_system_t *vesis_system;

void vesis_default_params(vesis_params *p);
void vesis_default_relax_opts(vesis_relax_opts *o);

/* Creates a system: copies the atom data to the device and allocates the
 * scratch for its grid (about 40 bytes per cell plus per-atom buffers).
 * Eq. (freeenergyfn), (G_VISM), (LJpotential), (Gss).
 *   xyz       n_atoms x 3 positions (must lie inside the box)
 *   sigma_sw, eps_sw  solute-solvent LJ parameters of each atom (A, kBT)
 *   q         partial charges (e)
 *   sigma_ss, eps_ss  solute-solute LJ parameters; a pair uses
 *             (sigma_i + sigma_j)/2 and sqrt(eps_i eps_j)
 *   bonds     n_bonds x 2 atom indices; harmonic 1/2 A (r - r0)^2 with
 *             A = bond_k, r0 = bond_r0; bonded pairs are excluded from
 *             the non-bonded terms (at most 8 bonds per atom)
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default)
 * n_atoms >= 1, n_bonds >= 0.  On error *out is NULL. */
int vesis_init_system(const vesis_params *p, int n_atoms, const double *xyz,
                      const double *sigma_sw, const double *eps_sw,
                      const double *q, const double *sigma_ss,
                      const double *eps_ss, int n_bonds, const int *bonds,
                      const double *bond_k, const double *bond_r0,
                      void *cuda_stream, vesis_system *out);

/* Replaces the atom positions (n_atoms x 3, host). */
int vesis_set_positions(vesis_system s, const double *xyz);

/* Copies the current positions (n_atoms x 3) to host memory. */
int vesis_get_positions(vesis_system s, double *xyz_out);

/* Initial labels (Sec. 3.1, "Initial surfaces"):
 *   kind 0: loose sphere, chi = 1 where |x - center| < radius;
 *   kind 1: tight surface, chi = 1 where min_i (|x - r_i| - d_i) < 0 at
 *           the cell centre, d = n_atoms radii (host; NULL: sigma_sw).
 * chi_dev: G bytes, written. */
int vesis_init_labels(vesis_system s, int kind, const double *d,
                      double radius, const double *center, uint8_t *chi_dev);

/* Energy density and Coulomb field on every cell (Eq. Ur):
 *   U = rho_w sum_i U_LJ^(i)(r) + C |E|^2,  E = sum_i Q_i d / r^3,
 *   C = (l_B / 8 pi)(1/eps_w - 1/eps_m),  d = x - r_i,  r = max(|d|, r_min).
 * xyz_or_null: new positions (host, n_atoms x 3) or NULL for the current.
 * U_dev: G floats; E_dev: 3 x G floats (Ex block, Ey block, Ez block) or
 * NULL.  FP32 pair sums.  If chi_dev is not NULL and terms_out is not NULL,
 * terms_out[0..5] = surface, vdW, CFA, far field, solute-solute, total
 * (FP64; vdW and CFA need E_dev). */
int vesis_energy_field(vesis_system s, const double *xyz_or_null,
                       float *U_dev, float *E_dev, const uint8_t *chi_dev,
                       double *terms_out);

/* Energy terms of a labelled state from given fields (Eq. 4flip plus the
 * far field and G_ss at the current positions):
 *   surface = c sum_j chi_j (1 - w_j) = c_N sum_j chi_j (S - W_j) with W
 *             the integer kernel convolution of chi and S the sum of the
 *             kernel's weights (either kernel; see vesis_params.kernel),
 *   volume  = h^3 sum_{chi_j = 0} U_j  (split into vdW and CFA if E_dev).
 * terms_out[6] as for vesis_energy_field. */
int vesis_energy_terms(vesis_system s, const uint8_t *chi_dev,
                       const float *U_dev, const float *E_dev,
                       double *terms_out);

/* Kernel convolution of the labels (Eq. Area), exact integers, cells
 * outside the box solvent: with the separable Gaussian W_dev[j] = 256^3 w_j
 * (<= 2^24); with the sin^2 kernel W_dev[j] = sum_k round(2^16 K_jk) chi_k.
 * G uint32, written. */
int vesis_surface_weights(vesis_system s, const uint8_t *chi_dev,
                          uint32_t *W_dev);

/* Flip energies (Eq. dGj1 / dGj2 with the h^3 of the centre-point rule):
 *   dE_j = c [s_j (1 - 2 w_j) - g0] - s_j h^3 U_j,  s_j = 1 - 2 chi_j,
 * w = W / S, g0 = the centre weight / S, evaluated in FP64 on candidate
 * cells (a face neighbour with the other label) as c_N N_j - s_j h^3 U_j
 * with the exact integer N_j = s_j (S - 2 W_j) - centre weight.
 * dE_dev: G doubles (0 on non-candidates); cand_dev: G bytes. */
int vesis_flip_energies(vesis_system s, const uint8_t *chi_dev,
                        const float *U_dev, double *dE_dev,
                        uint8_t *cand_dev);

/* Binary level-set relaxation at fixed atoms (Sec. 3.1, Step 2): rounds
 * of flips until no candidate lowers the energy - the data-parallel form of
 * the min-heap flipping.  A candidate with dE < 0 has the key (float(dE),
 * then index); with r the kernel's half-width in cells (trunc_r, or the
 * sin^2 kernel's radius), the grid is cut into bricks of edge 4 (edge 2
 * when r < 3) and a brick's leader is its smallest key; each round flips
 * every leader that no other leader within Chebyshev distance r precedes.
 * The heap's top always flips, flipped cells are more than r apart, and a
 * round lowers the energy by exactly the sum of their dE.
 *   chi_dev   G bytes, relaxed in place
 *   U_dev     G floats from vesis_energy_field at the current positions
 *   E_dev     3 x G floats or NULL (only for the vdW/CFA split of terms)
 *   max_rounds  > 0
 * Outputs (each may be NULL): rounds with flips, flipped cells, the sum of
 * the flipped cells' dE (FP64), terms[6] of the relaxed state.
 * Returns VESIS_W_MAX_ROUNDS if the cap stopped it. */
int vesis_blsm_relax(vesis_system s, uint8_t *chi_dev, const float *U_dev,
                     const float *E_dev, int max_rounds, int *rounds_out,
                     long long *flips_out, double *dE_sum_out,
                     double *terms_out);

/* vesis_blsm_relax of many systems in one persistent launch: the flip
 * rounds of every system run in the same cooperative kernel, whose blocks
 * serve the 8^3 tiles of all systems round-robin, with one grid barrier
 * per phase for all of them.  Each system goes through exactly the rounds
 * it would go through alone (same labels, rounds and flips; the FP64 sum of
 * its flipped dE is added in another fixed order, so it may differ from
 * vesis_blsm_relax's in the last bits), and its W is left as the exact
 * convolution of its relaxed labels.  The paper relaxes one solute at a
 * time (Sec. 3.3); this serves many solutes, for example the plain
 * relaxations a learned initialiser is trained on.
 *   nsys       1..64 distinct systems on one device with the same surface
 *              kernel (kind, half-width and weights; for the sin^2 kernel
 *              the same h and lambda)
 *   chi_dev[i] system i's labels, relaxed in place; U_dev[i] its energy
 *              density (vesis_energy_field)
 *   max_rounds > 0, the cap on the rounds of the launch
 * Outputs (each may be NULL, else nsys entries): each system's rounds with
 * flips, flipped cells and FP64 sum of their dE.  Every system's stream is
 * waited for; the work runs on systems[0]'s stream, and the call returns
 * when it is done.  Returns VESIS_W_MAX_ROUNDS if the cap stopped any
 * system.  Device scratch for the launch (about 300 bytes per system) is
 * allocated and freed by the call. */
int vesis_blsm_relax_batch(int nsys, vesis_system *systems, uint8_t *const *chi_dev,
                           const float *const *U_dev, int max_rounds, int *rounds_out,
                           long long *flips_out, double *dE_sum_out);

/* The paper's literal serial flipping (Sec. 3.1, Steps 2.1-2.2) on the
 * GPU: of the cells next to the interface (a face neighbour with the other
 * label) with dE < 0, flip the one with the smallest dE (ties: smaller
 * linear index), update w and dE in its kernel window and the candidate
 * set, and repeat until no candidate has dE < 0 or max_flips flips were
 * made.  The order is the min-heap's; the smallest key is kept in a
 * tournament of 4^3 tiles and groups of 8^3 tiles, run by one block (the
 * process is serial, so it runs at one flip every few microseconds, far
 * slower than vesis_blsm_relax on large grids).  Same arguments as
 * vesis_blsm_relax; max_flips >= 0.  The call also stops after 16 G + 1024
 * flips: a guard against a cycle of flips whose FP64 dE rounds below zero.
 * Outputs (each may be NULL): flips, the FP64 sum of the flipped cells' dE
 * in flip order, terms[6] of the relaxed state.
 * Returns VESIS_W_MAX_ROUNDS if max_flips stopped it. */
int vesis_blsm_heap(vesis_system s, uint8_t *chi_dev, const float *U_dev,
                    const float *E_dev, long long max_flips, long long *flips_out,
                    double *dE_sum_out, double *terms_out);

/* Gradient dG/dr_n of the total free energy with the interface fixed
 * (Eq. GradientG, taken as the exact derivative of the discrete energy):
 * grid term -h^3 sum over solvent cells, far-field term and G_ss.
 *   chi_dev      labels (G bytes)
 *   xyz_or_null  positions to evaluate at (host) or NULL for the current
 *   E_dev        3 x G field at those positions, or NULL to compute it
 *   grad_out     host, n_atoms x 3 FP64
 *   energy_out   host, total G at that state (may be NULL) */
int vesis_atom_forces(vesis_system s, const uint8_t *chi_dev,
                      const double *xyz_or_null, const float *E_dev,
                      double *grad_out, double *energy_out);

/* Full VESIS relaxation (Sec. 3.3, Steps 1-5) from chi_dev and xyz_inout:
 * flips to a local minimum (Step 2), gradient test (Step 3.2), forward
 * Euler step with M_nl = omega M, omega = 1 / max |dG/dr| (Eq. adjustmml),
 * accept or shrink M (Step 3.4), energy test held for `window` steps
 * (Steps 4-5).  chi_dev and xyz_inout are updated; stats_out may be NULL.
 * opts NULL means the defaults. */
int vesis_relax(vesis_system s, uint8_t *chi_dev, double *xyz_inout,
                const vesis_relax_opts *opts, vesis_relax_stats *stats_out);

/* Bound on the flip sweep's device-side waits.  The sweep (the rounds of
 * vesis_blsm_relax and of the interface relaxations inside vesis_relax)
 * runs as one cooperative launch whose blocks meet at a grid barrier twice
 * per round.  A block that has polled the barrier `polls` times without
 * seeing it complete (each poll an L2 load plus a 32 ns sleep) raises the
 * sweep's error flag and returns, and so does every other block at its
 * next barrier; the call then returns VESIS_E_CUDA with the message "flip
 * sweep grid barrier timed out".  The labels passed in are then partly
 * relaxed and must be reset by the caller; the system stays usable, and
 * the next call starts its sweep state afresh.  Default 2^24 polls (seconds
 * of waiting: only a hung block reaches it).  polls >= 0; 0 gives up at the
 * first poll that finds the barrier still open, which makes the failure
 * path testable without any fault.  VESIS_E_ARG for polls < 0. */
int vesis_set_wait_limit(vesis_system s, long long polls);

/* Which tiles a round of the flip sweep decides.  A leader's verdict (Sec.
 * 3.1, Step 2, in the brick-leader form) depends only on the leader words
 * within r of it, so a tile none of whose 27 neighbouring tiles changed a
 * leader word in the previous round keeps its previous verdict (it lost)
 * and need not be decided again; the updates stamp the tiles whose
 * neighbourhood changed.  mode -1 (the default): stamps are written while
 * the tiles holding a leader outnumber the sweep's warps, and read by a
 * block whose own leader tiles outnumber its warps; 0: never (every tile
 * holding a leader is decided every round); 1: always.  The rounds,
 * flips, labels and energies are identical in every mode; only the time
 * differs.  Applies to later vesis_blsm_relax, vesis_relax and (through
 * the first system) vesis_blsm_relax_batch calls.  VESIS_E_ARG for another
 * mode or a NULL system. */
int vesis_set_sweep_stamps(vesis_system s, int mode);

/* Per-iteration log: every later vesis_relax on the system writes one
 * record per accepted outer iteration into records (host memory, kept by
 * the caller until the log is replaced or the system destroyed), the
 * first `capacity` of them; stats->records counts those written by a
 * call.  records = NULL or capacity = 0 turns the log off.  VESIS_E_ARG
 * for capacity < 0. */
int vesis_set_history(vesis_system s, vesis_iter_record *records, int capacity);

/* The system's relaxation state: written by every vesis_relax that ends
 * with status >= 0 (cleared to valid = 0 by one that fails), read by
 * vesis_relax with opts.resume = 1.  set checks that k, ncnt and stable
 * are >= 0 and M, G_prev finite with M > 0 (VESIS_E_ARG otherwise); a
 * state with valid = 0 is stored as given and makes a resume fail. */
int vesis_get_state(vesis_system s, vesis_relax_state *out);
int vesis_set_state(vesis_system s, const vesis_relax_state *st);

/* Tile shapes of the two pair kernels: cells of a z-pencil per thread of
 * the energy-density kernel (4, 8 or 16, default 8) and atoms per thread of the
 * grid-to-atom gradient kernel (2 or 4, default 4).  Every cell sums its
 * atoms, and every atom its cells, in the same order for all shapes, so
 * the results are bit-identical; only the time differs.  Waits for the
 * system's stream.  VESIS_E_ARG for any other value. */
int vesis_set_tiles(vesis_system s, int energy_pencil, int force_atoms);
int vesis_get_tiles(vesis_system s, int *energy_pencil, int *force_atoms);

/* Autotuner: times each tile shape of the two pair kernels on the system's
 * current positions and labels chi_dev (one warm-up and `reps` launches
 * each, 1..1000, CUDA events on the system's stream) and keeps the fastest
 * (vesis_set_tiles).  times_ms_out (may be NULL): 5 doubles, the mean
 * launch time of energy pencil 4, 8, 16 and gradient atoms 2, 4. */
int vesis_autotune(vesis_system s, const uint8_t *chi_dev, int reps,
                   double *times_ms_out);

/* Batched relaxation: vesis_relax of every system i on (chi_dev[i],
 * xyz_inout[i]) with the same opts, run by `threads` host threads (1..256)
 * that take the systems from a shared queue, largest grid x atoms first.
 * The paper relaxes one solute at a time; this is a service for many
 * small solutes.  Each system runs on a private non-blocking stream for
 * the call (its own stream is drained first and given back afterwards),
 * so one system's kernels overlap another's host steps and kernel tails.
 * The flip sweep is one cooperative launch whose blocks must be resident
 * together: at most `sweep_slots` (1..16) sweeps run at a time, each on
 * 1 / sweep_slots of the device's sweep blocks.  The results of every
 * system (labels, positions, stats) equal those of vesis_relax called on
 * it alone.  The systems must be distinct and on one device.
 *   stats_out  nsys entries or NULL;  status_out  nsys ints or NULL: each
 *              system's vesis_status
 * Returns VESIS_OK, or the first system's error (index in the message)
 * if any system failed; warnings are only reported in status_out. */
int vesis_relax_batch(int nsys, vesis_system *systems, uint8_t *const *chi_dev,
                      double *const *xyz_inout, const vesis_relax_opts *opts,
                      int threads, int sweep_slots, vesis_relax_stats *stats_out,
                      int *status_out);

/* ------------------------------------------------------------------------
 * Learned initialiser.  The paper starts the flips from a tight or a loose
 * surface (Sec. 3.1, "Initial surfaces"); this library can instead start
 * from the guess of a small 3-D U-Net of the relaxed labels, after which
 * the unchanged flip sweep finishes (so the sweep is both the fallback and
 * the measure of the guess's error).  Network: channels 32, 64, 128, 128 on
 * four levels (full, 1/2, 1/4, 1/8 resolution), one 3x3x3 conv + ReLU per
 * level and per decoder level, 2x2x2 mean pooling, nearest doubling with
 * skip concatenation, 1x1x1 head giving the logit of chi = 1; loss the mean
 * binary cross entropy.  BF16 weights and activations, FP32 accumulation
 * on the tensor cores; FP32 master weights trained by Adam.
 *
 * Features (vesis_features): three FP32 planes of the grid, in this order:
 * asinh((U - C|E|^2) / scale) (the vdW part of the energy density),
 * asinh(C|E|^2 / scale) (the CFA part), and the tight-surface labels (the
 * atom-density indicator: 1 within sigma_i of an atom).
 *
 * Parameters: one flat FP32 vector, layer by layer (e0, e1, e2, e3, d2,
 * d1, d0, head), each W[cout][cin][3][3][3] (1x1x1 for the head) then
 * b[cout]; cin of e0 = n_features, of d2/d1/d0 = skip + coarse channels. */
typedef struct vesis_net_t *vesis_net;

/* Creates a network for n_features (1..32) input planes with all
 * parameters zero; work goes on cuda_stream (NULL = legacy default). */
int vesis_net_create(int n_features, void *cuda_stream, vesis_net *out);
int vesis_net_param_count(vesis_net n, long long *count);
/* Host FP32 parameter vectors (param_count floats); set clears Adam's
 * moments and step. */
int vesis_net_set_params(vesis_net n, const float *theta);
int vesis_net_get_params(vesis_net n, float *theta);

/* Logits of a crop of a grid.  x_dev: n_features FP32 planes of the whole
 * NX x NY x NZ grid (plane-major, cell index (i*NY + j)*NZ + k).  crop:
 * {ox, oy, oz, cx, cy, cz} (each cx, cy, cz a positive multiple of 8,
 * inside the grid) or NULL for the whole grid (then NX, NY, NZ must be
 * multiples of 8).  logit_dev: cx*cy*cz floats or NULL; chi_dev: the same
 * number of bytes, the guess chi = [logit > 0], or NULL. */
int vesis_net_forward(vesis_net n, const float *x_dev, int NX, int NY, int NZ,
                      const int *crop, float *logit_dev, uint8_t *chi_dev);

/* Loss (mean binary cross entropy against chi_dev, the labels of the whole
 * grid, read in the crop) and its gradient with respect to the parameters,
 * kept for vesis_net_adam_step and copied to grad_host (param_count floats)
 * if it is not NULL. */
int vesis_net_loss_grad(vesis_net n, const float *x_dev, const uint8_t *chi_dev,
                        int NX, int NY, int NZ, const int *crop, double *loss_out,
                        float *grad_host);

/* Convolution kernels: kind 0 = mma.sync (BF16 tensor-core instructions
 * issued per warp), kind 1 = tcgen05 (5th-generation tensor cores, FP32
 * accumulators in tensor memory) wherever a level's grid has ny % 16 == 0
 * and nz % 8 == 0, kind 0 elsewhere (the default is 1).  Both give the
 * same sums up to FP32 rounding order. */
int vesis_net_set_conv_kernel(vesis_net n, int kind);

/* One Adam step with the last gradient (bias-corrected moments). */
int vesis_net_adam_step(vesis_net n, double lr, double beta1, double beta2, double eps);
int vesis_net_destroy(vesis_net n);

/* Solute-solute terms at the current positions (Eq. Gss), to FP64
 * accuracy (pair terms in double-float arithmetic, sums in FP64): out5[0]
 * bonds, [1] Lennard-Jones, [2] Coulomb, [3] bends, [4] torsions (their
 * sum is terms[4] of the energy calls).  The potential of mean force of
 * the paper's appendix needs the pair parts apart. */
int vesis_ss_terms(vesis_system s, double *out5);

/* Bending and torsion terms of G_ss (Eq. Gss), replacing any set before
 * (n_angles = n_torsions = 0 removes them; a new system has none):
 *   bend (i, j, k):  1/2 B (theta - theta0)^2, theta the angle between
 *                    r_i - r_j and r_k - r_j; ijk [n_angles][3], B and
 *                    theta0 (radians, in [0, pi]) n_angles each
 *   torsion (i, j, k, l): sum_{n=0..6} C_n [1 + cos(n tau - psi_n)], tau
 *                    the angle between (r_j - r_i) x (r_k - r_j) and
 *                    (r_k - r_j) x (r_l - r_k); ijkl [n_torsions][4], C and
 *                    psi [n_torsions][7]; each psi_n 0 or pi (the paper's
 *                    force formulas of the appendix assume so)
 * Their energies join terms[4] and their gradients (the appendix's) the
 * atom gradient.  A bend with sin theta = 0 adds no gradient; a torsion
 * whose two plane normals has a zero vector adds nothing.  Atoms of a term
 * must be distinct and in range.  Host arrays, copied. */
int vesis_set_bonded(vesis_system s, int n_angles, const int *ijk, const double *B,
                     const double *theta0, int n_torsions, const int *ijkl,
                     const double *C, const double *psi);

/* Features of the learned initialiser for a system: U_dev and E_dev from
 * vesis_energy_field at the current positions, chi_tight_dev the tight
 * labels (vesis_init_labels kind 1); x_dev: 3 x G floats, written.
 * scale > 0 (kBT/A^3). */
int vesis_features(vesis_system s, const float *U_dev, const float *E_dev,
                   const uint8_t *chi_tight_dev, double scale, float *x_dev);

/* Device time of the hot kernels, measured with CUDA events recorded on the
 * system's stream around each launch while timing is enabled. */
typedef struct {
    double pair_energy_ms;       /* grid energy-density kernel */
    long long pair_energy_launches;
    long long pair_energy_pairs; /* cells x atoms over those launches */
    double pair_force_ms;        /* grid -> atom gradient kernel */
    long long pair_force_launches;
    long long pair_force_pairs;  /* solvent cells x atoms */
    double sweep_ms;             /* flip-round batches (all round kernels) */
    long long sweep_rounds;      /* rounds enqueued in those batches */
    long long sweep_cells;       /* cells x rounds enqueued */
    long long kernel_launches;   /* library kernels launched (all systems) */
    double conv_ms;              /* surface-kernel convolutions (three passes each) */
    long long conv_launches;     /* convolutions timed */
    long long conv_cells;        /* cells x convolutions */
    long long sweep_tiles_decide;   /* 8^3 tiles visited by the sweeps' decide
                                       phases (a tile holding a leader, per round) */
    long long sweep_tiles_update;   /* and by their update phases (a tile a
                                       winner reached, per round) */
} vesis_timing;

/* enable != 0 starts recording (and clears the totals); 0 stops. */
int vesis_set_timing(vesis_system s, int enable);

/* Synchronises the stream and returns the totals since timing was enabled. */
int vesis_get_timing(vesis_system s, vesis_timing *out);

/* Largest grid (cells) vesis_surface_weights_noalloc accepts. */
#define VESIS_NOALLOC_MAX_CELLS (1 << 20)

/* The kernel convolution of vesis_surface_weights for the separable
 * Gaussian (W_dev[j] = 256^3 w_j, exact; p->kernel must be 0) for callers
 * that cannot allocate device memory.  The paper has no
 * counterpart: it is a service of this library.  Creating a vesis_system
 * calls cudaMalloc; code running while a stream is captured into a CUDA
 * graph, processes whose device memory belongs to a pool or arena that
 * forbids other allocations, and loops that must not enter the driver's
 * allocator cannot do that.  This call needs no system and allocates
 * nothing itself: its two intermediate planes live in a fixed array of
 * device global memory (6 bytes per cell for VESIS_NOALLOC_MAX_CELLS
 * cells, about 6 MiB) that a GPU reserves when it loads the library's
 * module and holds until the process exits.  Under CUDA's default lazy
 * module loading that happens at the first call on the device (with
 * CUDA_MODULE_LOADING=EAGER, when the library is loaded), so callers whose
 * memory a pool or arena takes over must make that first call before it
 * does.
 *   p        grid (nx, ny, nz), h, gauss_sigma and trunc_r are used; at most
 *            VESIS_NOALLOC_MAX_CELLS cells, larger grids return VESIS_E_ARG
 *   chi_dev  G labels (device), W_dev G uint32 (device, written)
 *   cuda_stream  stream to enqueue on (NULL = legacy default); the call
 *            returns once the work is enqueued
 * Each call whose stream is not being captured looks up the array's device
 * address (with that device current); during a capture the address from
 * the last such call on the device is used, so the first call on a device
 * must come before any stream capture (one made during a capture returns
 * VESIS_E_ARG).
 * All calls share the one array, and each call writes it in full before
 * reading it: calls whose work overlaps on the GPU (other streams, other
 * threads) race and must be serialised by the caller. */
int vesis_surface_weights_noalloc(const vesis_params *p, const uint8_t *chi_dev,
                                  uint32_t *W_dev, void *cuda_stream);

/* Frees the system's device memory.  NULL is accepted. */
int vesis_destroy(vesis_system s);

/* Message of the last error on this thread ("" if none). */
const char *vesis_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VESIS_H */
