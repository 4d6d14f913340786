// Internal declarations of the VESIS CUDA library (sm_103a).
// Shared by the library's translation units only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vesis {

constexpr int kMaxR = 8;  // largest kernel half-width in cells

// Grid geometry in box-centred FP32 coordinates: the centre of cell i on
// an axis with n cells is (i - (n - 1)/2) h, exact up to one rounding.
struct GridDesc {
    int nx, ny, nz;
    float h;
    float cx, cy, cz;  // (n - 1) / 2 per axis
};

__device__ __forceinline__ float cell_pos(int i, float half, float h) {
    return ((float)i - half) * h;
}

// Integer 1-D weights q[a + r], a = -r..r, of the product surface kernel.
struct KernelW {
    int r;
    int q[2 * kMaxR + 1];
};

// Device views of the atom data (box-centred FP32 coordinates).
struct AtomsDev {
    int n;
    const float4 *xyzq;   // x, y, z, Q
    const float2 *ab;     // A = 4 eps sigma^12, B = 4 eps sigma^6
    const float4 *fcoef;  // 12 rho_w A, -6 rho_w B, -2 C Q, 0
};

// Per-relaxation flip-round state, in device memory.
struct RoundState {
    int done;              // 1 once a round flips nothing or the cap is hit
    int round;             // rounds that flipped cells
    int capped;            // 1 if max_rounds stopped the rounds
    int max_rounds;
    unsigned long long round_flips;   // flips of the round in progress
    unsigned long long total_flips;
    double round_dE;       // sum of dE of the round in progress
    double total_dE;
    unsigned long long tiles_decide;   // 8^3 tiles visited by the decide phases
    unsigned long long tiles_update;   // and by the update phases
};

// Counts kernel launches made by the library (reported by the timing API).
void count_launch(int n = 1);
long long launch_count();

// ---------------------------------------------------------------- pair.cu
// pts: cells of a z-pencil per thread (4 or 8; equal sums either way)
void launch_pair_energy_grid(const GridDesc &g, const AtomsDev &a, float rho,
                             float cfa, float rmin2, float *U, float *Ex,
                             float *Ey, float *Ez, int pts, cudaStream_t st);
// Far-field nodes: pts[k] = (x, y, z, _); writes U, E per node and the
// FP64 partial sums of w_k U_k per block into part (nblocks doubles).
int point_energy_blocks(int np);
void launch_point_energy(const float4 *pts, const double *w, int np,
                         const AtomsDev &a, float rho, float cfa, float rmin2,
                         float4 *UE, double *part, cudaStream_t st);
// Grid -> atom gradient partials: part[chunk][atom][3] (FP64); the solvent
// cells visited are added to *nsolvent (may be NULL).
struct ForcePlan {
    int nchunk;
    long long chunk_len;
    int atom_tiles;
    int apt;          // atoms per thread of the grid kernel (2 or 4)
    int cg;           // cell groups of a block: 128 / cg threads hold the tile's atoms,
                      // and each group takes every cg-th cell of a stage (1, 2 or 4)
};
ForcePlan plan_pair_force(long long G, int natoms, int nsm, int apt);
void launch_pair_force_grid(const GridDesc &g, const ForcePlan &fp,
                            const uint8_t *chi, const float *Ex,
                            const float *Ey, const float *Ez,
                            const AtomsDev &a, float rmin2, double *part,
                            unsigned long long *nsolvent, cudaStream_t st);
// Point-list (far-field) gradient partials: part[chunk][atom][3].
ForcePlan plan_point_force(int np, int natoms, int nsm);
void launch_point_force(const float4 *pts, const float *wf, int np,
                        const float4 *UE, const ForcePlan &fp,
                        const AtomsDev &a, float rmin2, double *part,
                        cudaStream_t st);
// Sum of partials in chunk order, scaled: out[n*3+l] (FP64).
void launch_force_reduce(const double *part, int nchunk, int natoms,
                         double scale, double *out, int accumulate,
                         cudaStream_t st);
// Ordered sum of `n` doubles (single block) into out[0] (optionally added).
void launch_sum_doubles(const double *in, int n, double *out, int accumulate,
                        cudaStream_t st);

// ---------------------------------------------------------------- blsm.cu
// Exact integer passes of the separable surface kernel: T1 = z pass of chi
// (<= 256), T2 = y pass of T1 (<= 2^16), W = x pass of T2 (<= 2^24).
void launch_conv_z(const GridDesc &g, const KernelW &kw, const uint8_t *chi,
                   uint16_t *T1, cudaStream_t st);
void launch_conv_y(const GridDesc &g, const KernelW &kw, const uint16_t *T1,
                   uint32_t *T2, cudaStream_t st);
void launch_conv_x(const GridDesc &g, const KernelW &kw, const uint32_t *T2,
                   uint32_t *W, cudaStream_t st);
// W = the direct convolution of chi with a full integer stencil k3 of
// (2R+1)^3 weights (device, centred: offset (a,b,c) at ((a+R)(2R+1) + b+R)
// (2R+1) + c+R), for the sin^2 kernel that is not a product.
void launch_conv3(const GridDesc &g, int R, const int *k3, const uint8_t *chi,
                  uint32_t *W, cudaStream_t st);
// Flip energy dE = cN N - s h3 U with the exact integer N = s (S - 2W) - k0
// (S: sum of all kernel weights, k0: centre weight; Eq. dGj1/dGj2).
struct FlipConst {
    double cN, h3;
    int S, k0;
};
// Face neighbour with the other label; outside the box counts as solvent.
__device__ __forceinline__ bool is_candidate(const GridDesc &g,
                                             const uint8_t *__restrict__ chi,
                                             long long p, int i, int j, int k,
                                             long long nyz)
{
    const uint8_t c = chi[p];
    const uint8_t xm = (i > 0) ? chi[p - nyz] : 0;
    const uint8_t xp = (i < g.nx - 1) ? chi[p + nyz] : 0;
    const uint8_t ym = (j > 0) ? chi[p - g.nz] : 0;
    const uint8_t yp = (j < g.ny - 1) ? chi[p + g.nz] : 0;
    const uint8_t zm = (k > 0) ? chi[p - 1] : 0;
    const uint8_t zp = (k < g.nz - 1) ? chi[p + 1] : 0;
    return (xm != c) | (xp != c) | (ym != c) | (yp != c) | (zm != c) | (zp != c);
}

// dE of Eq. (dGj1/dGj2): c [s (1 - 2w) - g0] - s h^3 U with w = W / S and
// g0 = k0 / S is cN N - s h^3 U for the exact integer N = s (S - 2W) - k0
// and cN = c / S; both products are rounded once and the sum once (no
// contraction).
__device__ __forceinline__ double flip_dE(uint8_t chi_j, unsigned W, float U,
                                          const FlipConst &fc)
{
    const int base = fc.S - 2 * (int)W;
    const int N = (chi_j ? -base : base) - fc.k0;
    const double t1 = __dmul_rn(fc.cN, (double)N);
    const double t2 = __dmul_rn(fc.h3, (double)U);
    return __dadd_rn(t1, chi_j ? t2 : -t2);
}

void launch_flip_energy(const GridDesc &g, const uint32_t *W,
                        const uint8_t *chi, const float *U, const FlipConst &fc,
                        double *dE, uint8_t *cand, cudaStream_t st);
// Energy sums over a labelled grid: per-block partials then ordered final.
int terms_blocks(long long G);
// ksum: sum of all kernel weights (S above); part_s collects sum chi (S - W).
void launch_terms(const GridDesc &g, const uint8_t *chi, const uint32_t *W,
                  const float *U, const float *Ex, const float *Ey,
                  const float *Ez, float cfa, unsigned ksum, long long *part_s,
                  double *part_v, double *part_c, cudaStream_t st);
// out[0] = c * S / D^3, out[1] = h^3 * sum U (solvent), out[2] = h^3 * sum
// C|E|^2 (solvent), out[3] = number of solute cells.
void launch_terms_final(const long long *part_s, const double *part_v,
                        const double *part_c, int nb, double c, double D3,
                        double h3, double *out, cudaStream_t st);
void launch_init_sphere(const GridDesc &g, float cx, float cy, float cz,
                        float radius, uint8_t *chi, cudaStream_t st);
void launch_init_tight(const GridDesc &g, const float4 *xyzd, int n,
                       uint8_t *chi, cudaStream_t st);

// --------------------------------------------------------------- sweep.cu
// Persistent narrow-band flip sweep: all rounds in one cooperative launch.
int sweep_tiles(const GridDesc &g);
int sweep_brick_edge(int r);
long long sweep_bricks(const GridDesc &g, int r);
cudaError_t sweep_grid_size(int nsm, int r, int *blocks);
int sweep_ctl_words();   // unsigned words of the sweep control block
// Bytes of sweep state (leader words, per-tile postings and flags).
size_t sweep_state_bytes(const GridDesc &g, int r);
// dE: G doubles, state: sweep_state_bytes(), ctl: sweep_ctl_words(),
// err: 1 int, part_flips and part_dE: `blocks` entries, part_tiles: 2 x
// `blocks` (tiles visited by the decide and update phases); k3: the full stencil (device,
// (2 kw.r + 1)^3, centred) or NULL for the product kernel kw.q; writes the
// totals into *rs.
// Bends and torsions of G_ss (atoms.cu): term lists and, per atom, the
// terms it takes part in (entry = term << 2 | role, role = its position in
// the term).
struct BondedDev {
    int nang = 0, ntor = 0;
    const int *ang = nullptr;       // [nang][3]
    const double *angB = nullptr, *angT0 = nullptr;
    const int *tor = nullptr;       // [ntor][4]
    const double *torC = nullptr, *torPsi = nullptr;   // [ntor][7]
    const int *ang_ptr = nullptr, *ang_inc = nullptr;  // CSR over atoms
    const int *tor_ptr = nullptr, *tor_inc = nullptr;
};
// Energies (ordered sums) into e_bend and e_tors; grad (if not NULL) += the
// terms' gradient; part: nang + ntor doubles of scratch.
void launch_bonded(const BondedDev &b, const double *xyz, int n, double *part, double *e_bend,
                   double *e_tors, double *grad, cudaStream_t st);
// Input features of the learned initialiser (unet.cu): three FP32 planes
// asinh((U - cfa |E|^2) / scale), asinh(cfa |E|^2 / scale), chi_t.
void launch_features(const float *U, const float *E, long long G, const uint8_t *chi_t,
                     float cfa, float scale, float *x, cudaStream_t st);
// The literal serial flipping (heap.cu): key = G doubles of scratch,
// state = heap_state_bytes(g) bytes; the counts land in flips_out,
// dsum_out and capped_out (device).
size_t heap_state_bytes(const GridDesc &g);
cudaError_t launch_heap(const GridDesc &g, const KernelW &kw, const int *k3,
                        const FlipConst &fc, uint8_t *chi, uint32_t *W, const float *U,
                        double *key, void *state, long long max_flips, long long *flips_out,
                        double *dsum_out, int *capped_out, cudaStream_t st);
cudaError_t launch_sweep(const GridDesc &g, const KernelW &kw, const int *k3,
                         const FlipConst &fc,
                         uint8_t *chi, uint32_t *W, const float *U,
                         double *dE, void *state, unsigned *ctl, int *err,
                         unsigned long long *part_flips, double *part_dE,
                         unsigned long long *part_tiles,
                         int *rounds, int *capped, int max_rounds, int blocks,
                         long long spin_limit, int stamps, RoundState *rs, cudaStream_t st);
// Decide stamps of the sweep (which tiles a round's decide visits): -1
// while the leader tiles outnumber the grid's warps, 0 never (every leader
// tile is decided every round), 1 always.  The rounds and labels are the
// same in every mode.
// Default bound on a sweep block's polls of its grid barrier (several
// seconds of waiting).
constexpr long long kSweepSpinLimit = 1ll << 24;
// Multi-system sweep: the rounds of up to kMaxSweepSys systems (same
// surface kernel) in one cooperative launch.  Per system: its grid, flip
// constants, labels, W, U, dE scratch, sweep state, control words and
// error flag (as for launch_sweep), a per-tile FP64 dE sum and flip count
// (sweep_tiles(g) entries each), its RoundState and the stream its
// set-up is enqueued on.  scratch: sweep_multi_scratch_bytes(nsys) bytes
// of device memory; err_out (pinned host, may be NULL) receives the
// launch's error flag.  Everything else is enqueued on st.
constexpr int kMaxSweepSys = 64;
struct SweepSys {
    GridDesc g;
    FlipConst fc;
    uint8_t *chi;
    uint32_t *W;
    const float *U;
    double *dE;
    void *state;
    unsigned *ctl;
    int *err;
    double *tile_dE;
    unsigned *tile_nf;
    RoundState *rs;
    cudaStream_t st;
};
size_t sweep_multi_scratch_bytes(int nsys);
cudaError_t launch_sweep_multi(int nsys, const SweepSys *sys, const KernelW &kw, const int *k3,
                               int max_rounds, int blocks, long long spin_limit, int stamps,
                               void *scratch, int *err_out, cudaStream_t st);

// --------------------------------------------------------------- atoms.cu
struct AtomParamsDev {
    const double *sig_sw, *eps_sw, *q;   // per atom, FP64
};
// Packs FP64 positions (relative to the box centre) into the FP32 views.
void launch_pack_atoms(const double *xyz, const double *centre,
                       const double *sig, const double *eps, const double *q,
                       int n, double rho, double cfa, float4 *xyzq,
                       float2 *ab, float4 *fcoef, int *oob, const double *lo,
                       const double *hi, cudaStream_t st);
// Solute-solute energy and gradient to FP64 accuracy (Eq. Gss; pair terms
// in double-float arithmetic) on a 2-D grid of
// (atom tile, j-chunk) blocks: e_part[block][3] (bond, LJ, Coulomb) and
// g_part[chunk][n][3] (gradient partials, summed in chunk order later).
struct SsPlan {
    int tiles, nchunk, chunk_len;
};
SsPlan plan_ss(int n, int nsm);
void launch_ss(const SsPlan &sp, const double *xyz, const double *sig,
               const double *sqeps, const double *q, const int *excl,
               const int *bond_ptr, const int *bond_other, const double *bond_k,
               const double *bond_r0, int n, double coul, double *e_part,
               double *g_part, cudaStream_t st);
void launch_ss_final(const double *e_part, int nb, double *out3,
                     cudaStream_t st);
// grad = a + b (+ c), and the max |component| into *gmax (FP64 bits).
void launch_grad_combine(const double *a, const double *b, double *grad,
                         int n3, unsigned long long *gmax_bits,
                         cudaStream_t st);
// xyz_new = xyz - (M / gmax) grad (Eq. moveatoms, Eq. adjustmml).
void launch_mobility(const double *xyz, const double *grad,
                     const unsigned long long *gmax_bits, const double *M,
                     double *xyz_new, int n3, cudaStream_t st);

}  // namespace vesis
