// C ABI of the VESIS hot path (include/vesis.h): system set-up, orchestration
// of the kernels on the caller's stream, and the relaxation loop of
// Sec. 3.3 (Steps 1-5) with its accept/shrink test run on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "vesis.h"
#include "vesis_internal.cuh"

using namespace vesis;

namespace {
// NVTX range over a scope: the phases of a relaxation show up by name in a
// profiler's timeline (no cost without one attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

#include <atomic>

namespace vesis {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace vesis

namespace {

thread_local std::string g_err;

}  // namespace

namespace vesis {
// The calling thread's error message slot (also used by noalloc.cu).
std::string *noalloc_last_error() { return &g_err; }
}  // namespace vesis

namespace {

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define VCK(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return fail(VESIS_E_CUDA, std::string(#call) + ": " +              \
                                          cudaGetErrorString(e_));             \
    } while (0)

// Device scalar slots of an energy bank.
enum {
    S_SURF = 0, S_VOL = 1, S_CFA = 2, S_NSOL = 3, S_FAR = 4,
    S_SSB = 5, S_SSLJ = 6, S_SSC = 7, S_TOTAL = 8, S_SSA = 9, S_SST = 10, S_BANK = 16
};

struct GdState {
    double M;
    int ncnt;
    int decision;   // 0 accept, 1 reject, 2 the gradient test ends the relaxation
    double dG;
};

__global__ void k_total(double *bank)
{
    bank[S_TOTAL] = bank[S_SURF] + bank[S_VOL] + bank[S_FAR] + bank[S_SSB] +
                    bank[S_SSLJ] + bank[S_SSC] + bank[S_SSA] + bank[S_SST];
}

// Step 3.4: reject if dG > dG* or (N_cnt >= N*_cnt and 0 < dG <= dG*), with
// dG* = frac |G_old|; a rejection shrinks M by alpha and resets N_cnt, an
// acceptance increments N_cnt.  A non-finite trial energy or an atom that
// left the box is rejected like an energy increase.
// Step 3.4's accept/shrink test of a trial step.  The first trial of an
// iteration is enqueued before the host has seen the gradient: when Step
// 3.2's test (max |dG/dr| below Tol1, or not finite) ends the relaxation
// instead, the trial is void and M and N_cnt are left as they are.
__global__ void k_gd_decide(GdState *s, const double *bank_old,
                            const double *bank_new, const int *oob,
                            int ncnt_star, double frac, double alpha,
                            const unsigned long long *gmax_bits, double tol_grad)
{
    const double gmax = __longlong_as_double((long long)*gmax_bits);
    if (!(gmax == gmax) || gmax >= 1.0e308 || gmax < tol_grad) {
        s->decision = 2;
        return;
    }
    const double Gold = bank_old[S_TOTAL], Gnew = bank_new[S_TOTAL];
    const double dG = Gnew - Gold;
    const double dGs = frac * fabs(Gold);
    bool reject = (dG > dGs) || (s->ncnt >= ncnt_star && dG > 0.0 && dG <= dGs);
    if (!(Gnew == Gnew) || *oob) reject = true;
    if (reject) {
        s->M *= alpha;
        s->ncnt = 0;
        s->decision = 1;
    } else {
        s->ncnt += 1;
        s->decision = 0;
    }
    s->dG = dG;
}

__global__ void k_gd_init(GdState *s, double M0, int ncnt0)
{
    s->M = M0;
    s->ncnt = ncnt0;
    s->decision = 0;
    s->dG = 0.0;
}

// Gauss-Legendre nodes and weights on (-1, 1): Newton iteration on the
// three-term recurrence of the Legendre polynomials.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p0 = 1.0;
                p1 = z;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace

// Admission of flip sweeps while several systems relax at once: each sweep
// is one cooperative launch whose blocks must all be resident together, so
// at most `slots` sweeps run at a time and each uses `blocks` blocks, with
// slots x blocks no more than one wave of the device.  Other kernels always
// end by themselves, so an admitted sweep only waits for them to drain.
struct SweepGate {
    std::mutex m;
    std::condition_variable cv;
    int free_slots = 1;
    int blocks = 1;
    void acquire()
    {
        std::unique_lock<std::mutex> l(m);
        cv.wait(l, [&] { return free_slots > 0; });
        --free_slots;
    }
    void release()
    {
        {
            std::lock_guard<std::mutex> l(m);
            ++free_slots;
        }
        cv.notify_one();
    }
};

struct vesis_system_t {
    int dev = 0;
    cudaStream_t st = nullptr;
    int nsm = 152;
    vesis_params p{};
    int n = 0;
    GridDesc g{};
    long long G = 0;
    KernelW kw{};
    FlipConst fc{};
    int *d_k3 = nullptr;        // full stencil of the sin^2 kernel, or NULL
    long long ksum = 0;         // sum of all kernel weights
    double terms_c = 0, terms_D = 1;   // E_s = terms_c * sum chi (S - W) / terms_D
    double c = 0, g0 = 0, h3 = 0, cfa = 0, lB = 0, coul = 0;
    float rmin2 = 0.f;
    double centre[3]{}, lo[3]{}, hi[3]{};
    std::vector<double> sig_sw;

    double *d_xyz = nullptr, *d_xyz_new = nullptr;
    double *d_sig_sw = nullptr, *d_eps_sw = nullptr, *d_q = nullptr;
    double *d_sig_ss = nullptr, *d_sqeps_ss = nullptr;
    double *d_geo = nullptr;   // centre[3], lo[3], hi[3]
    float4 *d_xyzq = nullptr, *d_fcoef = nullptr, *d_xyzd = nullptr;
    float2 *d_ab = nullptr;
    int *d_oob = nullptr;
    int *d_excl = nullptr, *d_bond_ptr = nullptr, *d_bond_other = nullptr;
    double *d_bond_k = nullptr, *d_bond_r0 = nullptr;

    uint16_t *d_T1 = nullptr;
    uint32_t *d_T2 = nullptr, *d_W = nullptr;
    double *d_dE = nullptr;
    float *d_U[2] = {nullptr, nullptr}, *d_E[2] = {nullptr, nullptr};

    long long *d_part_s = nullptr;
    double *d_part_v = nullptr, *d_part_c = nullptr;
    int nb_terms = 0;
    ForcePlan fplan{}, fplan_far{};
    int pe_pts = 8;             // cells per thread of the energy kernel (4 or 8)
    SweepGate *gate = nullptr;  // set while a batched relaxation runs
    double *d_fpart = nullptr;
    double *d_grad_solv = nullptr, *d_grad_ss = nullptr, *d_grad = nullptr;
    unsigned long long *d_gmax = nullptr;
    unsigned long long *d_fcount = nullptr;   // solvent cells seen by forces

    int nfar = 0;
    float4 *d_far_pts = nullptr, *d_far_UE = nullptr;
    double *d_far_w = nullptr, *d_far_part = nullptr;
    float *d_far_wf = nullptr;
    int nb_far = 0;

    double *d_ss_part = nullptr, *d_ss_gpart = nullptr;
    BondedDev bonded{};               // bends and torsions (none by default)
    double *d_bonded_part = nullptr;
    std::vector<void *> bonded_allocs;
    int nb_ss = 0;
    SsPlan ssplan{};

    // persistent sweep state
    int sweep_blocks = 0, ntiles = 0;
    long long spin_limit = kSweepSpinLimit;   // polls of a sweep barrier wait
    int sweep_stamps = -1;                    // decide stamps of the sweep (-1, 0, 1)
    uint8_t *d_sweep = nullptr;
    uint8_t *d_heap = nullptr;      // tile and group keys of the serial flipping
    long long *d_heap_out = nullptr;   // flips, dE sum (as bits), capped
    unsigned *d_ctl = nullptr;
    int *d_err = nullptr, *d_rounds = nullptr, *d_capped = nullptr;
    unsigned long long *d_part_flips = nullptr;
    double *d_part_dE = nullptr;
    unsigned long long *d_part_tiles = nullptr;
    double *d_tile_dE = nullptr;      // multi-system sweep: per-tile dE sums
    unsigned *d_tile_nf = nullptr;    // and flip counts

    double *d_scal = nullptr;   // two banks of S_BANK doubles
    RoundState *d_rs = nullptr;
    GdState *d_gd = nullptr;
    vesis_relax_state rstate{};   // where the last relaxation stopped
    vesis_iter_record *hist = nullptr;   // caller's per-iteration log (host)
    int hist_cap = 0;

    // pinned host mirrors
    double *h_scal = nullptr;
    double *h_scal2 = nullptr;    // a second bank (the trial's, read with the current one)
    RoundState *h_rs = nullptr;
    GdState *h_gd = nullptr;
    int *h_int = nullptr;
    unsigned long long *h_u64 = nullptr;

    std::vector<void *> allocs;

    // optional event timing of the hot kernels
    bool timing = false;
    struct Span {
        cudaEvent_t a, b;
        int kind;            // 0 energy, 1 force, 2 sweep batch
        long long units;     // pairs or cells x rounds
        long long rounds;
        long long tiles_decide, tiles_update;   // sweep: tiles visited per phase
    };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> ev_pool;
    vesis_timing tm{};
    long long launches0 = 0;
};

namespace {

template <typename T>
int dalloc(vesis_system s, T **ptr, size_t count)
{
    void *p = nullptr;
    const cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess)
        return fail(VESIS_E_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    s->allocs.push_back(p);
    *ptr = (T *)p;
    return VESIS_OK;
}

#define VTRY(x)                  \
    do {                         \
        int rc_ = (x);           \
        if (rc_ != VESIS_OK) {   \
            return rc_;          \
        }                        \
    } while (0)

cudaEvent_t take_event(vesis_system s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Opens a timed span on the stream (no-op unless timing is enabled).
int span_begin(vesis_system s)
{
    if (!s->timing) return -1;
    vesis_system_t::Span sp{take_event(s), take_event(s), 0, 0, 0, 0, 0};
    cudaEventRecord(sp.a, s->st);
    s->spans.push_back(sp);
    return (int)s->spans.size() - 1;
}

void span_end(vesis_system s, int id, int kind, long long units, long long rounds)
{
    if (id < 0) return;
    vesis_system_t::Span &sp = s->spans[id];
    sp.kind = kind;
    sp.units = units;
    sp.rounds = rounds;
    cudaEventRecord(sp.b, s->st);
}

// Folds completed spans into the totals (the stream must be synchronised).
void collect_spans(vesis_system s)
{
    for (auto &sp : s->spans) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, sp.a, sp.b);
        if (sp.kind == 0) {
            s->tm.pair_energy_ms += ms;
            s->tm.pair_energy_launches += 1;
            s->tm.pair_energy_pairs += sp.units;
        } else if (sp.kind == 1) {
            s->tm.pair_force_ms += ms;
            s->tm.pair_force_launches += 1;
            s->tm.pair_force_pairs += sp.units;
        } else if (sp.kind == 2) {
            s->tm.sweep_ms += ms;
            s->tm.sweep_rounds += sp.rounds;
            s->tm.sweep_cells += sp.units;
            s->tm.sweep_tiles_decide += sp.tiles_decide;
            s->tm.sweep_tiles_update += sp.tiles_update;
        } else {
            s->tm.conv_ms += ms;
            s->tm.conv_launches += 1;
            s->tm.conv_cells += sp.units;
        }
        s->ev_pool.push_back(sp.a);
        s->ev_pool.push_back(sp.b);
    }
    s->spans.clear();
}

AtomsDev atoms_view(vesis_system s)
{
    AtomsDev a;
    a.n = s->n;
    a.xyzq = s->d_xyzq;
    a.ab = s->d_ab;
    a.fcoef = s->d_fcoef;
    return a;
}

double *bank(vesis_system s, int b) { return s->d_scal + b * S_BANK; }

void enq_pack(vesis_system s, const double *d_pos)
{
    cudaMemsetAsync(s->d_oob, 0, sizeof(int), s->st);
    launch_pack_atoms(d_pos, s->d_geo, s->d_sig_sw, s->d_eps_sw, s->d_q, s->n,
                      s->p.rho_w, s->cfa, s->d_xyzq, s->d_ab, s->d_fcoef,
                      s->d_oob, s->d_geo + 3, s->d_geo + 6, s->st);
}

// Far-field energy and node fields at the packed positions.
void enq_far(vesis_system s, double *bk)
{
    if (s->nfar > 0) {
        launch_point_energy(s->d_far_pts, s->d_far_w, s->nfar, atoms_view(s),
                            (float)s->p.rho_w, (float)s->cfa, s->rmin2,
                            s->d_far_UE, s->d_far_part, s->st);
        launch_sum_doubles(s->d_far_part, s->nb_far, bk + S_FAR, 0, s->st);
    } else {
        cudaMemsetAsync(bk + S_FAR, 0, sizeof(double), s->st);
    }
}

void enq_fields(vesis_system s, float *U, float *E, double *bk)
{
    const int sp = span_begin(s);
    launch_pair_energy_grid(s->g, atoms_view(s), (float)s->p.rho_w,
                            (float)s->cfa, s->rmin2, U, E, E + s->G,
                            E + 2 * s->G, s->pe_pts, s->st);
    span_end(s, sp, 0, s->G * (long long)s->n, 0);
    enq_far(s, bk);
}

void enq_ss(vesis_system s, const double *d_pos, double *bk)
{
    launch_ss(s->ssplan, d_pos, s->d_sig_ss, s->d_sqeps_ss, s->d_q, s->d_excl,
              s->d_bond_ptr, s->d_bond_other, s->d_bond_k, s->d_bond_r0, s->n,
              s->coul, s->d_ss_part, s->d_ss_gpart, s->st);
    launch_ss_final(s->d_ss_part, s->nb_ss, bk + S_SSB, s->st);
    launch_force_reduce(s->d_ss_gpart, s->ssplan.nchunk, s->n, 1.0, s->d_grad_ss,
                        0, s->st);
    launch_bonded(s->bonded, d_pos, s->n, s->d_bonded_part, bk + S_SSA, bk + S_SST,
                  s->d_grad_ss, s->st);
}

void enq_conv(vesis_system s, const uint8_t *chi, uint32_t *W)
{
    const int sp = span_begin(s);
    if (s->d_k3) {
        launch_conv3(s->g, s->kw.r, s->d_k3, chi, W, s->st);
    } else {
        launch_conv_z(s->g, s->kw, chi, s->d_T1, s->st);
        launch_conv_y(s->g, s->kw, s->d_T1, s->d_T2, s->st);
        launch_conv_x(s->g, s->kw, s->d_T2, W, s->st);
    }
    span_end(s, sp, 3, s->G, 0);
}

// Surface and volume terms of a labelled state; total with far and ss slots.
// w_current: d_W already holds the exact convolution of chi (the flip sweep
// keeps it so), and the three passes are skipped.
void enq_terms(vesis_system s, const uint8_t *chi, const float *U,
               const float *E, double *bk, bool w_current = false)
{
    if (!w_current) enq_conv(s, chi, s->d_W);
    launch_terms(s->g, chi, s->d_W, U, E, E ? E + s->G : nullptr,
                 E ? E + 2 * s->G : nullptr, (float)s->cfa, (unsigned)s->ksum,
                 s->d_part_s, s->d_part_v, s->d_part_c, s->st);
    launch_terms_final(s->d_part_s, s->d_part_v, s->d_part_c, s->nb_terms,
                       s->terms_c, s->terms_D, s->h3, bk, s->st);
    count_launch();
    k_total<<<1, 1, 0, s->st>>>(bk);
}

// The flip sweep to a local minimum.  defer: the sweep's record and error
// flag are copied out but not waited for; the caller waits with its next
// read and then calls finish_blsm (not with a sweep gate: a gated sweep
// holds its slot until it has ended).
int finish_blsm(vesis_system s, int sp, RoundState *out);
int run_blsm(vesis_system s, uint8_t *chi, const float *U, int max_rounds,
             RoundState *out, bool w_current = false, int *defer_sp = nullptr)
{
    // exact integer convolution of the starting labels (unless d_W holds it
    // already); the sweep keeps it current with every flip
    if (!w_current) enq_conv(s, chi, s->d_W);
    // batched: the stream is drained first so that an admitted sweep starts
    // at once, and the slot is held until the sweep has ended
    struct Hold {
        SweepGate *g;
        ~Hold()
        {
            if (g) g->release();
        }
    } hold{nullptr};
    int blocks = s->sweep_blocks;
    if (s->gate) {
        VCK(cudaStreamSynchronize(s->st));
        s->gate->acquire();
        hold.g = s->gate;
        blocks = std::max(1, std::min(blocks, s->gate->blocks));
    }
    const int sp = span_begin(s);
    VCK(launch_sweep(s->g, s->kw, s->d_k3, s->fc, chi, s->d_W, U, s->d_dE, s->d_sweep,
                     s->d_ctl, s->d_err, s->d_part_flips,
                     s->d_part_dE, s->d_part_tiles, s->d_rounds, s->d_capped, max_rounds,
                     blocks, s->spin_limit, s->sweep_stamps, s->d_rs, s->st));
    span_end(s, sp, 2, 0, 0);
    VCK(cudaMemcpyAsync(s->h_rs, s->d_rs, sizeof(RoundState),
                        cudaMemcpyDeviceToHost, s->st));
    VCK(cudaMemcpyAsync(s->h_int, s->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                        s->st));
    if (defer_sp && !s->gate) {
        *defer_sp = sp;
        return VESIS_OK;
    }
    VCK(cudaStreamSynchronize(s->st));
    if (defer_sp) *defer_sp = -2;    // already finished
    return finish_blsm(s, sp, out);
}

// The sweep's outcome once its copies have landed (after a synchronisation).
int finish_blsm(vesis_system s, int sp, RoundState *out)
{
    if (*s->h_int) return fail(VESIS_E_CUDA, "flip sweep grid barrier timed out");
    if (sp >= 0) {
        // the rounds include the last one, which found nothing to flip
        const long long rounds = s->h_rs->round + (s->h_rs->capped ? 0 : 1);
        s->spans[sp].rounds = rounds;
        s->spans[sp].units = s->G * rounds;
        s->spans[sp].tiles_decide = (long long)s->h_rs->tiles_decide;
        s->spans[sp].tiles_update = (long long)s->h_rs->tiles_update;
    }
    *out = *s->h_rs;
    return VESIS_OK;
}

// Gradient at the packed positions; E: the 3 x G field there.  Requires the
// far-field node fields of the same positions (enq_far).  Writes d_grad and
// d_gmax, and the solute-solute energies into bk.  ss_current: the last
// enq_ss ran at d_pos into bk (its gradient is still in d_grad_ss), so the
// solute-solute terms are not evaluated again.
void enq_gradient(vesis_system s, const uint8_t *chi, const float *E,
                  const double *d_pos, double *bk, bool ss_current = false)
{
    const int sp = span_begin(s);
    launch_pair_force_grid(s->g, s->fplan, chi, E, E + s->G, E + 2 * s->G,
                           atoms_view(s), s->rmin2, s->d_fpart, s->d_fcount,
                           s->st);
    span_end(s, sp, 1, 0, 0);
    launch_force_reduce(s->d_fpart, s->fplan.nchunk, s->n, s->h3,
                        s->d_grad_solv, 0, s->st);
    if (s->nfar > 0) {
        launch_point_force(s->d_far_pts, s->d_far_wf, s->nfar, s->d_far_UE,
                           s->fplan_far, atoms_view(s), s->rmin2, s->d_fpart,
                           s->st);
        launch_force_reduce(s->d_fpart, s->fplan_far.nchunk, s->n, 1.0,
                            s->d_grad_solv, 1, s->st);
    }
    if (!ss_current) enq_ss(s, d_pos, bk);
    launch_grad_combine(s->d_grad_solv, s->d_grad_ss, s->d_grad, 3 * s->n,
                        s->d_gmax, s->st);
}

int read_bank(vesis_system s, const double *bk)
{
    VCK(cudaMemcpyAsync(s->h_scal, bk, S_BANK * sizeof(double),
                        cudaMemcpyDeviceToHost, s->st));
    VCK(cudaStreamSynchronize(s->st));
    return VESIS_OK;
}

void fill_terms(const double *hb, bool have_E, double *terms)
{
    const double vol = hb[S_VOL];
    const double cfa = have_E ? hb[S_CFA] : 0.0;
    terms[0] = hb[S_SURF];
    terms[1] = vol - cfa;
    terms[2] = cfa;
    terms[3] = hb[S_FAR];
    terms[4] = hb[S_SSB] + hb[S_SSLJ] + hb[S_SSC] + hb[S_SSA] + hb[S_SST];
    terms[5] = hb[S_TOTAL];
}

int check_oob(vesis_system s)
{
    VCK(cudaMemcpyAsync(s->h_int, s->d_oob, sizeof(int), cudaMemcpyDeviceToHost,
                        s->st));
    VCK(cudaStreamSynchronize(s->st));
    if (*s->h_int) return fail(VESIS_E_OUT_OF_BOX, "an atom lies outside the box");
    return VESIS_OK;
}

int upload_xyz(vesis_system s, const double *xyz, double *dst)
{
    VCK(cudaMemcpyAsync(dst, xyz, 3 * sizeof(double) * s->n,
                        cudaMemcpyHostToDevice, s->st));
    // the source may be pageable; make the copy complete before returning
    VCK(cudaStreamSynchronize(s->st));
    return VESIS_OK;
}

int last_launch(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(VESIS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return VESIS_OK;
}

}  // namespace

extern "C" {

void vesis_default_params(vesis_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->gamma0 = 0.174;
    p->rho_w = 0.0333;
    p->eps_m = 1.0;
    p->eps_w = 80.0;
    p->temperature = 298.0;
    p->eps_ss = 1.0;
    p->nx = p->ny = p->nz = 64;
    p->h = 0.25;
    p->origin[0] = p->origin[1] = p->origin[2] = -8.0;
    p->gauss_sigma = 0.0;
    p->trunc_r = 6;
    p->r_min = 0.2;
    p->far_field = 1;
    p->far_nuv = 16;
    p->far_nt = 8;
    p->kernel = 0;
    p->sin2_lambda = 2.0;
}

void vesis_default_relax_opts(vesis_relax_opts *o)
{
    if (!o) return;
    o->max_outer = 3000;
    o->ncnt_star = 5;
    o->window = 100;
    o->M0 = 1.0;
    o->alpha = 1.0 / std::sqrt(2.0);
    o->dgstar_frac = 0.05;
    o->tol_grad = 1e-4;
    o->tol_energy = 1e-5;
    o->max_flip_rounds = 100000;
    o->max_gd_retries = 60;
    o->resume = 0;
}

const char *vesis_last_error(void) { return g_err.c_str(); }

int vesis_set_timing(vesis_system s, int enable)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    VCK(cudaStreamSynchronize(s->st));
    collect_spans(s);
    s->timing = enable != 0;
    if (enable) {
        std::memset(&s->tm, 0, sizeof(s->tm));
        s->launches0 = launch_count();
        VCK(cudaMemsetAsync(s->d_fcount, 0, sizeof(unsigned long long), s->st));
        VCK(cudaStreamSynchronize(s->st));
    }
    return VESIS_OK;
}

int vesis_get_timing(vesis_system s, vesis_timing *out)
{
    if (!s || !out) return fail(VESIS_E_ARG, "NULL argument");
    VCK(cudaMemcpyAsync(s->h_u64, s->d_fcount, sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s->st));
    VCK(cudaStreamSynchronize(s->st));
    collect_spans(s);
    *out = s->tm;
    out->pair_force_pairs = (long long)(*s->h_u64) * s->n;
    out->kernel_launches = launch_count() - s->launches0;
    return VESIS_OK;
}

int vesis_destroy(vesis_system s)
{
    if (!s) return VESIS_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(s->dev);
    cudaStreamSynchronize(s->st);
    for (auto &sp : s->spans) {
        cudaEventDestroy(sp.a);
        cudaEventDestroy(sp.b);
    }
    for (auto e : s->ev_pool) cudaEventDestroy(e);
    for (void *p : s->allocs) cudaFree(p);
    for (void *p : s->bonded_allocs) cudaFree(p);
    if (s->h_scal) cudaFreeHost(s->h_scal);
    if (s->h_scal2) cudaFreeHost(s->h_scal2);
    if (s->h_rs) cudaFreeHost(s->h_rs);
    if (s->h_gd) cudaFreeHost(s->h_gd);
    if (s->h_int) cudaFreeHost(s->h_int);
    if (s->h_u64) cudaFreeHost(s->h_u64);
    cudaSetDevice(dev);
    delete s;
    return VESIS_OK;
}

static int init_impl(vesis_system s, const vesis_params *p, int n,
                     const double *xyz, const double *sigma_sw,
                     const double *eps_sw, const double *q,
                     const double *sigma_ss, const double *eps_ss, int nbond,
                     const int *bonds, const double *bond_k,
                     const double *bond_r0)
{
    s->p = *p;
    s->n = n;
    VCK(cudaGetDevice(&s->dev));
    VCK(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev));
    const long long G = (long long)p->nx * p->ny * p->nz;
    s->G = G;
    s->g.nx = p->nx;
    s->g.ny = p->ny;
    s->g.nz = p->nz;
    s->g.h = (float)p->h;
    s->g.cx = 0.5f * (float)(p->nx - 1);
    s->g.cy = 0.5f * (float)(p->ny - 1);
    s->g.cz = 0.5f * (float)(p->nz - 1);
    const int nn[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; ++d) {
        s->lo[d] = p->origin[d];
        s->hi[d] = p->origin[d] + nn[d] * p->h;
        s->centre[d] = p->origin[d] + 0.5 * nn[d] * p->h;
    }

    // physical constants (CODATA 2018) and the CFA prefactor of Eq. (Ur)
    const double e = 1.602176634e-19, eps0 = 8.8541878128e-12, kB = 1.380649e-23;
    s->lB = e * e / (4.0 * M_PI * eps0 * kB * p->temperature) * 1e10;
    s->cfa = s->lB / (8.0 * M_PI) * (1.0 / p->eps_w - 1.0 / p->eps_m);
    s->coul = s->lB / p->eps_ss;
    s->rmin2 = (float)(p->r_min * p->r_min);

    const double h = p->h;
    s->h3 = h * h * h;
    if (p->kernel == 1) {
        // the paper's sin^2 kernel (Sec. 3.1): weights round(2^16 sin^2(pi
        // rho / delta)) on the cells with rho = h |d| <= delta = lambda
        // sqrt(h); E_s = gamma0 C0 h^4 / lambda^4 sum over solute-solvent
        // pairs, C0 = 8 pi / (pi^2 - 3)
        const double lam = p->sin2_lambda;
        const double delta = lam * std::sqrt(h);
        const int R = (int)std::floor(delta / h);
        const int w = 2 * R + 1;
        std::vector<int> k3((size_t)w * w * w, 0);
        long long S = 0;
        for (int a = -R; a <= R; ++a)
            for (int b = -R; b <= R; ++b)
                for (int c = -R; c <= R; ++c) {
                    const double rho = h * std::sqrt((double)(a * a + b * b + c * c));
                    if (rho <= delta) {
                        const double v = std::sin(M_PI * rho / delta);
                        const int q = (int)std::nearbyint(65536.0 * (v * v));
                        k3[((size_t)(a + R) * w + (b + R)) * w + (c + R)] = q;
                        S += q;
                    }
                }
        const double C0 = 8.0 * M_PI / (M_PI * M_PI - 3.0);
        const double h4 = h * h * h * h;
        const double cN = ((p->gamma0 * C0) * h4) / (lam * lam * lam * lam * 65536.0);
        s->kw.r = R;
        s->ksum = S;
        s->fc.cN = cN;
        s->fc.h3 = s->h3;
        s->fc.S = (int)S;
        s->fc.k0 = k3[((size_t)R * w + R) * w + R];
        s->c = cN * (double)S;
        s->g0 = (double)s->fc.k0 / (double)S;
        s->terms_c = cN;
        s->terms_D = 1.0;
        VTRY(dalloc(s, &s->d_k3, k3.size()));
        VCK(cudaMemcpy(s->d_k3, k3.data(), k3.size() * sizeof(int), cudaMemcpyHostToDevice));
    } else {
        // separable Gaussian: integer 1-D weights summing to 256
        const double sig = p->gauss_sigma > 0.0 ? p->gauss_sigma : 2.0 * h;
        const int r = p->trunc_r;
        std::vector<double> gw(2 * r + 1);
        double gs = 0.0;
        for (int a = -r; a <= r; ++a) {
            gw[a + r] = std::exp(-(double)(a * a) / (2.0 * (sig / h) * (sig / h)));
            gs += gw[a + r];
        }
        int qsum = 0;
        s->kw.r = r;
        for (int a = -r; a <= r; ++a) {
            if (a == 0) continue;
            s->kw.q[a + r] = (int)std::nearbyint(256.0 * gw[a + r] / gs);
            qsum += s->kw.q[a + r];
        }
        s->kw.q[r] = 256 - qsum;
        if (s->kw.q[r] < 0) return fail(VESIS_E_ARG, "surface kernel weights exceed 256");
        long long S1 = 0;
        for (int a = 1; a <= r; ++a) S1 += (long long)a * s->kw.q[a + r];
        if (S1 <= 0) return fail(VESIS_E_ARG, "surface kernel has no first moment");
        s->c = p->gamma0 * h * h * 256.0 / (double)S1;
        const long long k0 = (long long)s->kw.q[r] * s->kw.q[r] * s->kw.q[r];
        s->g0 = (double)k0 / 16777216.0;
        s->ksum = 16777216;
        s->fc.cN = s->c / 16777216.0;
        s->fc.h3 = s->h3;
        s->fc.S = 16777216;
        s->fc.k0 = (int)k0;
        s->terms_c = s->c;
        s->terms_D = 16777216.0;
    }

    // atom data
    s->sig_sw.assign(sigma_sw, sigma_sw + n);
    std::vector<double> sqe(n);
    for (int i = 0; i < n; ++i) sqe[i] = std::sqrt(eps_ss[i]);
    VTRY(dalloc(s, &s->d_xyz, 3 * n));
    VTRY(dalloc(s, &s->d_xyz_new, 3 * n));
    VTRY(dalloc(s, &s->d_sig_sw, n));
    VTRY(dalloc(s, &s->d_eps_sw, n));
    VTRY(dalloc(s, &s->d_q, n));
    VTRY(dalloc(s, &s->d_sig_ss, n));
    VTRY(dalloc(s, &s->d_sqeps_ss, n));
    VTRY(dalloc(s, &s->d_geo, 9));
    VTRY(dalloc(s, &s->d_xyzq, n));
    VTRY(dalloc(s, &s->d_ab, n));
    VTRY(dalloc(s, &s->d_fcoef, n));
    VTRY(dalloc(s, &s->d_xyzd, n));
    VTRY(dalloc(s, &s->d_oob, 1));
    double geo[9] = {s->centre[0], s->centre[1], s->centre[2], s->lo[0], s->lo[1],
                     s->lo[2], s->hi[0], s->hi[1], s->hi[2]};
    VCK(cudaMemcpy(s->d_geo, geo, sizeof(geo), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_xyz, xyz, 3 * n * sizeof(double), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_sig_sw, sigma_sw, n * sizeof(double), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_eps_sw, eps_sw, n * sizeof(double), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_q, q, n * sizeof(double), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_sig_ss, sigma_ss, n * sizeof(double), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_sqeps_ss, sqe.data(), n * sizeof(double), cudaMemcpyHostToDevice));

    // bonds: per-atom exclusion lists and CSR bond lists
    constexpr int kMaxExcl = 8;
    std::vector<int> excl((size_t)n * kMaxExcl, -1), deg(n, 0);
    std::vector<int> ptr(n + 1, 0);
    for (int b = 0; b < nbond; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j)
            return fail(VESIS_E_ARG, "bond index out of range");
        if (deg[i] >= kMaxExcl || deg[j] >= kMaxExcl)
            return fail(VESIS_E_ARG, "more than 8 bonds on one atom");
        excl[(size_t)i * kMaxExcl + deg[i]++] = j;
        excl[(size_t)j * kMaxExcl + deg[j]++] = i;
    }
    for (int i = 0; i < n; ++i) ptr[i + 1] = ptr[i] + deg[i];
    std::vector<int> other(std::max(1, ptr[n]));
    std::vector<double> bk(std::max(1, ptr[n])), br(std::max(1, ptr[n]));
    std::vector<int> fillc(n, 0);
    for (int b = 0; b < nbond; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        int pi = ptr[i] + fillc[i]++, pj = ptr[j] + fillc[j]++;
        other[pi] = j; bk[pi] = bond_k[b]; br[pi] = bond_r0[b];
        other[pj] = i; bk[pj] = bond_k[b]; br[pj] = bond_r0[b];
    }
    VTRY(dalloc(s, &s->d_excl, (size_t)n * kMaxExcl));
    VTRY(dalloc(s, &s->d_bond_ptr, n + 1));
    VTRY(dalloc(s, &s->d_bond_other, other.size()));
    VTRY(dalloc(s, &s->d_bond_k, bk.size()));
    VTRY(dalloc(s, &s->d_bond_r0, br.size()));
    VCK(cudaMemcpy(s->d_excl, excl.data(), excl.size() * sizeof(int), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_bond_ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_bond_other, other.data(), other.size() * sizeof(int), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_bond_k, bk.data(), bk.size() * sizeof(double), cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(s->d_bond_r0, br.data(), br.size() * sizeof(double), cudaMemcpyHostToDevice));

    // grid scratch
    VTRY(dalloc(s, &s->d_T1, G));
    VTRY(dalloc(s, &s->d_T2, G));
    VTRY(dalloc(s, &s->d_W, G));
    VTRY(dalloc(s, &s->d_dE, G));
    for (int b = 0; b < 2; ++b) {
        VTRY(dalloc(s, &s->d_U[b], G));
        VTRY(dalloc(s, &s->d_E[b], 3 * G));
    }
    s->nb_terms = terms_blocks(G);
    VTRY(dalloc(s, &s->d_part_s, 2 * s->nb_terms));
    VTRY(dalloc(s, &s->d_part_v, s->nb_terms));
    VTRY(dalloc(s, &s->d_part_c, s->nb_terms));

    // far-field quadrature: six face pyramids about the box centre,
    // y = c + s p, s = 1/t >= 1, dV = Lx Ly Lz t^-4 dt du dv
    if (p->far_field) {
        std::vector<double> xu, wu, xt, wt;
        gauss_legendre(p->far_nuv, xu, wu);
        gauss_legendre(p->far_nt, xt, wt);
        const double Lh[3] = {0.5 * nn[0] * h, 0.5 * nn[1] * h, 0.5 * nn[2] * h};
        const double vol = Lh[0] * Lh[1] * Lh[2];
        std::vector<float4> pts;
        std::vector<double> w;
        std::vector<float> wf;
        for (int axis = 0; axis < 3; ++axis) {
            int oth[2], m = 0;
            for (int d = 0; d < 3; ++d)
                if (d != axis) oth[m++] = d;
            for (int sg = -1; sg <= 1; sg += 2)
                for (int iu = 0; iu < p->far_nuv; ++iu)
                    for (int iv = 0; iv < p->far_nuv; ++iv)
                        for (int it = 0; it < p->far_nt; ++it) {
                            const double t = 0.5 * (xt[it] + 1.0);
                            double f[3];
                            f[axis] = sg * Lh[axis];
                            f[oth[0]] = xu[iu] * Lh[oth[0]];
                            f[oth[1]] = xu[iv] * Lh[oth[1]];
                            const double ww = wu[iu] * wu[iv] * 0.5 * wt[it] * vol / (t * t * t * t);
                            pts.push_back(make_float4((float)(f[0] / t), (float)(f[1] / t),
                                                      (float)(f[2] / t), 0.f));
                            w.push_back(ww);
                            wf.push_back((float)ww);
                        }
        }
        s->nfar = (int)pts.size();
        VTRY(dalloc(s, &s->d_far_pts, s->nfar));
        VTRY(dalloc(s, &s->d_far_UE, s->nfar));
        VTRY(dalloc(s, &s->d_far_w, s->nfar));
        VTRY(dalloc(s, &s->d_far_wf, s->nfar));
        s->nb_far = point_energy_blocks(s->nfar);
        VTRY(dalloc(s, &s->d_far_part, s->nb_far));
        VCK(cudaMemcpy(s->d_far_pts, pts.data(), pts.size() * sizeof(float4), cudaMemcpyHostToDevice));
        VCK(cudaMemcpy(s->d_far_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
        VCK(cudaMemcpy(s->d_far_wf, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice));
    }

    // gradient partials
    s->fplan = plan_pair_force(G, n, s->nsm, 4);
    s->fplan_far = plan_point_force(std::max(1, s->nfar), n, s->nsm);
    const long long nch = std::max(s->fplan.nchunk, s->fplan_far.nchunk);
    VTRY(dalloc(s, &s->d_fpart, (size_t)nch * n * 3));
    VTRY(dalloc(s, &s->d_grad_solv, 3 * n));
    VTRY(dalloc(s, &s->d_grad_ss, 3 * n));
    VTRY(dalloc(s, &s->d_grad, 3 * n));
    VTRY(dalloc(s, &s->d_gmax, 1));
    VTRY(dalloc(s, &s->d_fcount, 1));
    VCK(cudaMemset(s->d_fcount, 0, sizeof(unsigned long long)));
    s->ssplan = plan_ss(n, s->nsm);
    s->nb_ss = s->ssplan.tiles * s->ssplan.nchunk;
    VTRY(dalloc(s, &s->d_ss_part, 3 * s->nb_ss));
    VTRY(dalloc(s, &s->d_ss_gpart, (size_t)3 * n * s->ssplan.nchunk));

    {
        const cudaError_t e = sweep_grid_size(s->nsm, s->kw.r, &s->sweep_blocks);
        if (e != cudaSuccess)
            return fail(VESIS_E_CUDA, std::string("sweep occupancy: ") + cudaGetErrorString(e));
    }
    s->ntiles = sweep_tiles(s->g);
    VTRY(dalloc(s, &s->d_sweep, sweep_state_bytes(s->g, s->kw.r)));
    VTRY(dalloc(s, &s->d_heap, heap_state_bytes(s->g)));
    VTRY(dalloc(s, &s->d_heap_out, 3));
    VTRY(dalloc(s, &s->d_ctl, sweep_ctl_words()));
    VTRY(dalloc(s, &s->d_err, 1));
    VTRY(dalloc(s, &s->d_rounds, 1));
    VTRY(dalloc(s, &s->d_capped, 1));
    VTRY(dalloc(s, &s->d_part_flips, s->sweep_blocks));
    VTRY(dalloc(s, &s->d_part_dE, s->sweep_blocks));
    VTRY(dalloc(s, &s->d_part_tiles, 2 * (size_t)s->sweep_blocks));
    VTRY(dalloc(s, &s->d_tile_dE, (size_t)s->ntiles));
    VTRY(dalloc(s, &s->d_tile_nf, (size_t)s->ntiles));

    VTRY(dalloc(s, &s->d_scal, 2 * S_BANK));
    VTRY(dalloc(s, &s->d_rs, 1));
    VTRY(dalloc(s, &s->d_gd, 1));
    VCK(cudaMemset(s->d_scal, 0, 2 * S_BANK * sizeof(double)));
    VCK(cudaMallocHost(&s->h_scal, S_BANK * sizeof(double)));
    VCK(cudaMallocHost(&s->h_scal2, S_BANK * sizeof(double)));
    VCK(cudaMallocHost(&s->h_rs, sizeof(RoundState)));
    VCK(cudaMallocHost(&s->h_gd, sizeof(GdState)));
    VCK(cudaMallocHost(&s->h_int, sizeof(int)));
    VCK(cudaMallocHost(&s->h_u64, sizeof(unsigned long long)));
    VCK(cudaDeviceSynchronize());
    return VESIS_OK;
}

int vesis_init_system(const vesis_params *p, int n, const double *xyz,
                      const double *sigma_sw, const double *eps_sw,
                      const double *q, const double *sigma_ss,
                      const double *eps_ss, int nbond, const int *bonds,
                      const double *bond_k, const double *bond_r0,
                      void *cuda_stream, vesis_system *out)
{
    if (!out) return fail(VESIS_E_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !xyz || !sigma_sw || !eps_sw || !q || !sigma_ss || !eps_ss)
        return fail(VESIS_E_ARG, "NULL parameter or atom array");
    if (n < 1) return fail(VESIS_E_ARG, "n_atoms must be >= 1");
    if (nbond < 0 || (nbond > 0 && (!bonds || !bond_k || !bond_r0)))
        return fail(VESIS_E_ARG, "bad bond arrays");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 4096 || p->ny > 4096 ||
        p->nz > 4096)
        return fail(VESIS_E_ARG, "grid dimensions must be in 1..4096");
    const long long G = (long long)p->nx * p->ny * p->nz;
    if (G > 2147483647LL) return fail(VESIS_E_ARG, "grid has more than 2^31-1 cells");
    if (!(p->h > 0.0)) return fail(VESIS_E_ARG, "h must be > 0");
    if (p->kernel != 0 && p->kernel != 1) return fail(VESIS_E_ARG, "kernel must be 0 or 1");
    if (p->kernel == 0 && (p->trunc_r < 1 || p->trunc_r > kMaxR))
        return fail(VESIS_E_ARG, "trunc_r must be in 1..8");
    if (p->kernel == 1) {
        if (!(p->sin2_lambda > 0.0)) return fail(VESIS_E_ARG, "sin2_lambda must be > 0");
        const double cells = p->sin2_lambda * std::sqrt(p->h) / p->h;
        if (!(cells >= 1.0 && cells < (double)(kMaxR + 1)))
            return fail(VESIS_E_ARG,
                        "sin^2 kernel radius lambda sqrt(h) must span 1..8 cells of h");
    }
    if (!(p->r_min > 0.0)) return fail(VESIS_E_ARG, "r_min must be > 0");
    if (!(p->temperature > 0.0) || !(p->eps_w > 0.0) || !(p->eps_m > 0.0) ||
        !(p->eps_ss > 0.0))
        return fail(VESIS_E_ARG, "temperature and permittivities must be > 0");
    if (p->far_field && (p->far_nuv < 1 || p->far_nt < 1 || p->far_nuv > 64 ||
                         p->far_nt > 64))
        return fail(VESIS_E_ARG, "far-field orders must be in 1..64");
    for (int i = 0; i < 3 * n; ++i)
        if (!std::isfinite(xyz[i])) return fail(VESIS_E_NAN, "non-finite position");
    vesis_system s = new vesis_system_t();
    s->st = (cudaStream_t)cuda_stream;
    int rc = init_impl(s, p, n, xyz, sigma_sw, eps_sw, q, sigma_ss, eps_ss,
                       nbond, bonds, bond_k, bond_r0);
    if (rc == VESIS_OK) {
        enq_pack(s, s->d_xyz);
        rc = check_oob(s);
    }
    if (rc != VESIS_OK) {
        std::string keep = g_err;
        vesis_destroy(s);
        g_err = keep;
        return rc;
    }
    *out = s;
    return VESIS_OK;
}

int vesis_set_positions(vesis_system s, const double *xyz)
{
    if (!s || !xyz) return fail(VESIS_E_ARG, "NULL argument");
    for (int i = 0; i < 3 * s->n; ++i)
        if (!std::isfinite(xyz[i])) return fail(VESIS_E_NAN, "non-finite position");
    VTRY(upload_xyz(s, xyz, s->d_xyz));
    enq_pack(s, s->d_xyz);
    return check_oob(s);
}

int vesis_get_positions(vesis_system s, double *xyz_out)
{
    if (!s || !xyz_out) return fail(VESIS_E_ARG, "NULL argument");
    VCK(cudaMemcpyAsync(xyz_out, s->d_xyz, 3 * sizeof(double) * s->n,
                        cudaMemcpyDeviceToHost, s->st));
    VCK(cudaStreamSynchronize(s->st));
    return VESIS_OK;
}

int vesis_init_labels(vesis_system s, int kind, const double *d, double radius,
                      const double *center, uint8_t *chi_dev)
{
    if (!s || !chi_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (kind == 0) {
        const double c0 = center ? center[0] : 0.0, c1 = center ? center[1] : 0.0,
                     c2 = center ? center[2] : 0.0;
        launch_init_sphere(s->g, (float)(c0 - s->centre[0]), (float)(c1 - s->centre[1]),
                           (float)(c2 - s->centre[2]), (float)radius, chi_dev, s->st);
    } else if (kind == 1) {
        std::vector<double> xyz(3 * s->n);
        VCK(cudaMemcpy(xyz.data(), s->d_xyz, xyz.size() * sizeof(double),
                       cudaMemcpyDeviceToHost));
        std::vector<float4> a(s->n);
        for (int i = 0; i < s->n; ++i)
            a[i] = make_float4((float)(xyz[3 * i] - s->centre[0]),
                               (float)(xyz[3 * i + 1] - s->centre[1]),
                               (float)(xyz[3 * i + 2] - s->centre[2]),
                               (float)(d ? d[i] : s->sig_sw[i]));
        VCK(cudaMemcpyAsync(s->d_xyzd, a.data(), a.size() * sizeof(float4),
                            cudaMemcpyHostToDevice, s->st));
        launch_init_tight(s->g, s->d_xyzd, s->n, chi_dev, s->st);
        VCK(cudaStreamSynchronize(s->st));
    } else {
        return fail(VESIS_E_ARG, "kind must be 0 (sphere) or 1 (tight)");
    }
    return last_launch("init_labels");
}

int vesis_energy_field(vesis_system s, const double *xyz, float *U_dev,
                       float *E_dev, const uint8_t *chi_dev, double *terms_out)
{
    if (!s || !U_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (xyz) VTRY(vesis_set_positions(s, xyz));
    else enq_pack(s, s->d_xyz);
    float *E = E_dev ? E_dev : s->d_E[0];
    double *bk = bank(s, 0);
    enq_fields(s, U_dev, E, bk);
    if (chi_dev && terms_out) {
        enq_ss(s, s->d_xyz, bk);
        enq_terms(s, chi_dev, U_dev, E_dev, bk);
        VTRY(last_launch("energy_field"));
        VTRY(read_bank(s, bk));
        fill_terms(s->h_scal, E_dev != nullptr, terms_out);
    } else {
        VTRY(last_launch("energy_field"));
        VCK(cudaStreamSynchronize(s->st));
    }
    return VESIS_OK;
}

int vesis_energy_terms(vesis_system s, const uint8_t *chi_dev, const float *U_dev,
                       const float *E_dev, double *terms_out)
{
    if (!s || !chi_dev || !U_dev || !terms_out) return fail(VESIS_E_ARG, "NULL argument");
    double *bk = bank(s, 0);
    enq_pack(s, s->d_xyz);
    enq_far(s, bk);
    enq_ss(s, s->d_xyz, bk);
    enq_terms(s, chi_dev, U_dev, E_dev, bk);
    VTRY(last_launch("energy_terms"));
    VTRY(read_bank(s, bk));
    fill_terms(s->h_scal, E_dev != nullptr, terms_out);
    return VESIS_OK;
}

int vesis_surface_weights(vesis_system s, const uint8_t *chi_dev, uint32_t *W_dev)
{
    if (!s || !chi_dev || !W_dev) return fail(VESIS_E_ARG, "NULL argument");
    enq_conv(s, chi_dev, W_dev);
    VTRY(last_launch("surface_weights"));
    VCK(cudaStreamSynchronize(s->st));
    return VESIS_OK;
}

int vesis_flip_energies(vesis_system s, const uint8_t *chi_dev, const float *U_dev,
                        double *dE_dev, uint8_t *cand_dev)
{
    if (!s || !chi_dev || !U_dev || !dE_dev || !cand_dev)
        return fail(VESIS_E_ARG, "NULL argument");
    enq_conv(s, chi_dev, s->d_W);
    launch_flip_energy(s->g, s->d_W, chi_dev, U_dev, s->fc, dE_dev, cand_dev, s->st);
    VTRY(last_launch("flip_energies"));
    VCK(cudaStreamSynchronize(s->st));
    return VESIS_OK;
}

int vesis_blsm_relax(vesis_system s, uint8_t *chi_dev, const float *U_dev,
                     const float *E_dev, int max_rounds, int *rounds_out,
                     long long *flips_out, double *dE_sum_out, double *terms_out)
{
    if (!s || !chi_dev || !U_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (max_rounds < 1) return fail(VESIS_E_ARG, "max_rounds must be >= 1");
    RoundState rs;
    VTRY(run_blsm(s, chi_dev, U_dev, max_rounds, &rs));
    VTRY(last_launch("blsm_relax"));
    if (rounds_out) *rounds_out = rs.round;
    if (flips_out) *flips_out = (long long)rs.total_flips;
    if (dE_sum_out) *dE_sum_out = rs.total_dE;
    if (terms_out) VTRY(vesis_energy_terms(s, chi_dev, U_dev, E_dev, terms_out));
    return rs.capped ? VESIS_W_MAX_ROUNDS : VESIS_OK;
}

int vesis_blsm_relax_batch(int nsys, vesis_system *systems, uint8_t *const *chi_dev,
                           const float *const *U_dev, int max_rounds, int *rounds_out,
                           long long *flips_out, double *dE_sum_out)
{
    if (nsys < 1 || nsys > kMaxSweepSys)
        return fail(VESIS_E_ARG, "nsys must be in 1.." + std::to_string(kMaxSweepSys));
    if (!systems || !chi_dev || !U_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (max_rounds < 1) return fail(VESIS_E_ARG, "max_rounds must be >= 1");
    vesis_system s0 = systems[0];
    for (int i = 0; i < nsys; ++i) {
        vesis_system s = systems[i];
        if (!s || !chi_dev[i] || !U_dev[i])
            return fail(VESIS_E_ARG, "NULL system or buffer at index " + std::to_string(i));
        for (int j = 0; j < i; ++j)
            if (systems[j] == s) return fail(VESIS_E_ARG, "a system appears twice in the batch");
        if (s->dev != s0->dev) return fail(VESIS_E_ARG, "systems are on different devices");
        bool same = s->kw.r == s0->kw.r && (s->d_k3 != nullptr) == (s0->d_k3 != nullptr);
        for (int a = 0; same && a <= 2 * s->kw.r; ++a) same = s->kw.q[a] == s0->kw.q[a];
        if (same && s->d_k3)
            same = s->p.h == s0->p.h && s->p.sin2_lambda == s0->p.sin2_lambda;
        if (!same) return fail(VESIS_E_ARG, "the systems' surface kernels differ");
    }
    int dev0 = 0;
    VCK(cudaGetDevice(&dev0));
    VCK(cudaSetDevice(s0->dev));
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{dev0};
    std::vector<SweepSys> ys((size_t)nsys);
    for (int i = 0; i < nsys; ++i) {
        vesis_system s = systems[i];
        enq_conv(s, chi_dev[i], s->d_W);
        SweepSys &y = ys[i];
        y.g = s->g;
        y.fc = s->fc;
        y.chi = chi_dev[i];
        y.W = s->d_W;
        y.U = U_dev[i];
        y.dE = s->d_dE;
        y.state = s->d_sweep;
        y.ctl = s->d_ctl;
        y.err = s->d_err;
        y.tile_dE = s->d_tile_dE;
        y.tile_nf = s->d_tile_nf;
        y.rs = s->d_rs;
        y.st = s->st;
    }
    void *scratch = nullptr;
    VCK(cudaMalloc(&scratch, sweep_multi_scratch_bytes(nsys)));
    struct Free {
        void *p;
        ~Free() { cudaFree(p); }
    } free_scratch{scratch};
    cudaStream_t st = s0->st;
    VCK(launch_sweep_multi(nsys, ys.data(), s0->kw, s0->d_k3, max_rounds, s0->sweep_blocks,
                           s0->spin_limit, s0->sweep_stamps, scratch, s0->h_int, st));
    VCK(cudaStreamSynchronize(st));
    if (*s0->h_int) return fail(VESIS_E_CUDA, "flip sweep grid barrier timed out");
    int rc = VESIS_OK;
    for (int i = 0; i < nsys; ++i) {
        vesis_system s = systems[i];
        VCK(cudaMemcpy(s->h_rs, s->d_rs, sizeof(RoundState), cudaMemcpyDeviceToHost));
        if (rounds_out) rounds_out[i] = s->h_rs->round;
        if (flips_out) flips_out[i] = (long long)s->h_rs->total_flips;
        if (dE_sum_out) dE_sum_out[i] = s->h_rs->total_dE;
        if (s->h_rs->capped) rc = VESIS_W_MAX_ROUNDS;
    }
    VTRY(last_launch("blsm_relax_batch"));
    return rc;
}

int vesis_blsm_heap(vesis_system s, uint8_t *chi_dev, const float *U_dev,
                    const float *E_dev, long long max_flips, long long *flips_out,
                    double *dE_sum_out, double *terms_out)
{
    if (!s || !chi_dev || !U_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (max_flips < 0) return fail(VESIS_E_ARG, "max_flips must be >= 0");
    // Each flip lowers the energy, so the process ends; the bound only
    // guards against a cycle of flips whose FP64 dE rounds below zero.
    const long long hard = 16 * s->G + 1024;
    enq_conv(s, chi_dev, s->d_W);
    long long *o = s->d_heap_out;
    VCK(launch_heap(s->g, s->kw, s->d_k3, s->fc, chi_dev, s->d_W, U_dev, s->d_dE, s->d_heap,
                    std::min(max_flips, hard), o, reinterpret_cast<double *>(o + 1),
                    reinterpret_cast<int *>(o + 2), s->st));
    VCK(cudaMemcpyAsync(s->h_scal, o, 3 * sizeof(long long), cudaMemcpyDeviceToHost, s->st));
    VCK(cudaStreamSynchronize(s->st));
    VTRY(last_launch("blsm_heap"));
    long long h[3];
    std::memcpy(h, s->h_scal, sizeof(h));
    double dsum;
    std::memcpy(&dsum, &h[1], sizeof(double));
    const int capped = (int)(h[2] & 0xffffffffll);
    if (flips_out) *flips_out = h[0];
    if (dE_sum_out) *dE_sum_out = dsum;
    if (terms_out) VTRY(vesis_energy_terms(s, chi_dev, U_dev, E_dev, terms_out));
    return capped ? VESIS_W_MAX_ROUNDS : VESIS_OK;
}

int vesis_ss_terms(vesis_system s, double *out5)
{
    if (!s || !out5) return fail(VESIS_E_ARG, "NULL argument");
    double *bk = bank(s, 1);
    enq_ss(s, s->d_xyz, bk);
    VTRY(last_launch("ss_terms"));
    VTRY(read_bank(s, bk));
    out5[0] = s->h_scal[S_SSB];
    out5[1] = s->h_scal[S_SSLJ];
    out5[2] = s->h_scal[S_SSC];
    out5[3] = s->h_scal[S_SSA];
    out5[4] = s->h_scal[S_SST];
    return VESIS_OK;
}

int vesis_set_bonded(vesis_system s, int n_angles, const int *ijk, const double *B,
                     const double *theta0, int n_torsions, const int *ijkl, const double *C,
                     const double *psi)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    if (n_angles < 0 || n_torsions < 0) return fail(VESIS_E_ARG, "negative term count");
    if (n_angles > 0 && (!ijk || !B || !theta0)) return fail(VESIS_E_ARG, "NULL angle array");
    if (n_torsions > 0 && (!ijkl || !C || !psi)) return fail(VESIS_E_ARG, "NULL torsion array");
    const int n = s->n;
    for (int m = 0; m < n_angles; ++m) {
        const int *t = ijk + 3 * m;
        for (int c = 0; c < 3; ++c)
            if (t[c] < 0 || t[c] >= n) return fail(VESIS_E_ARG, "angle atom index out of range");
        if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2])
            return fail(VESIS_E_ARG, "an angle repeats an atom");
        if (!std::isfinite(B[m]) || !std::isfinite(theta0[m]) || theta0[m] < 0.0 ||
            theta0[m] > M_PI)
            return fail(VESIS_E_ARG, "angle constants must be finite, theta0 in [0, pi]");
    }
    for (int m = 0; m < n_torsions; ++m) {
        const int *t = ijkl + 4 * m;
        for (int c = 0; c < 4; ++c)
            if (t[c] < 0 || t[c] >= n) return fail(VESIS_E_ARG, "torsion atom index out of range");
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (t[a] == t[b]) return fail(VESIS_E_ARG, "a torsion repeats an atom");
        for (int c = 0; c < 7; ++c) {
            const double ps = psi[7 * m + c];
            if (!std::isfinite(C[7 * m + c]) ||
                !(std::fabs(ps) < 1e-9 || std::fabs(ps - M_PI) < 1e-9))
                return fail(VESIS_E_ARG, "torsion phases must be 0 or pi, constants finite");
        }
    }
    VCK(cudaStreamSynchronize(s->st));
    for (void *p : s->bonded_allocs) cudaFree(p);
    s->bonded_allocs.clear();
    s->bonded = BondedDev{};
    s->d_bonded_part = nullptr;
    if (n_angles + n_torsions == 0) return VESIS_OK;
    // per-atom incidence lists, terms in increasing order
    std::vector<int> aptr(n + 1, 0), tptr(n + 1, 0);
    for (int m = 0; m < n_angles; ++m)
        for (int c = 0; c < 3; ++c) ++aptr[ijk[3 * m + c] + 1];
    for (int m = 0; m < n_torsions; ++m)
        for (int c = 0; c < 4; ++c) ++tptr[ijkl[4 * m + c] + 1];
    for (int a = 0; a < n; ++a) {
        aptr[a + 1] += aptr[a];
        tptr[a + 1] += tptr[a];
    }
    std::vector<int> ainc(std::max(1, aptr[n])), tinc(std::max(1, tptr[n]));
    {
        std::vector<int> fa(aptr.begin(), aptr.end() - 1), ft(tptr.begin(), tptr.end() - 1);
        for (int m = 0; m < n_angles; ++m)
            for (int c = 0; c < 3; ++c) ainc[fa[ijk[3 * m + c]]++] = (m << 2) | c;
        for (int m = 0; m < n_torsions; ++m)
            for (int c = 0; c < 4; ++c) tinc[ft[ijkl[4 * m + c]]++] = (m << 2) | c;
    }
    auto up = [&](const void *src, size_t bytes, void **dst) -> int {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess)
            return fail(VESIS_E_ALLOC, "device allocation failed");
        s->bonded_allocs.push_back(p);
        if (src && bytes && cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(VESIS_E_CUDA, "copy of the bonded terms failed");
        *dst = p;
        return VESIS_OK;
    };
    BondedDev b;
    b.nang = n_angles;
    b.ntor = n_torsions;
    void *q;
    VTRY(up(ijk, sizeof(int) * 3 * n_angles, &q)); b.ang = (const int *)q;
    VTRY(up(B, sizeof(double) * n_angles, &q)); b.angB = (const double *)q;
    VTRY(up(theta0, sizeof(double) * n_angles, &q)); b.angT0 = (const double *)q;
    VTRY(up(ijkl, sizeof(int) * 4 * n_torsions, &q)); b.tor = (const int *)q;
    VTRY(up(C, sizeof(double) * 7 * n_torsions, &q)); b.torC = (const double *)q;
    VTRY(up(psi, sizeof(double) * 7 * n_torsions, &q)); b.torPsi = (const double *)q;
    VTRY(up(aptr.data(), sizeof(int) * (n + 1), &q)); b.ang_ptr = (const int *)q;
    VTRY(up(ainc.data(), sizeof(int) * ainc.size(), &q)); b.ang_inc = (const int *)q;
    VTRY(up(tptr.data(), sizeof(int) * (n + 1), &q)); b.tor_ptr = (const int *)q;
    VTRY(up(tinc.data(), sizeof(int) * tinc.size(), &q)); b.tor_inc = (const int *)q;
    VTRY(up(nullptr, sizeof(double) * (n_angles + n_torsions), &q));
    s->d_bonded_part = (double *)q;
    s->bonded = b;
    return VESIS_OK;
}

int vesis_features(vesis_system s, const float *U_dev, const float *E_dev,
                   const uint8_t *chi_tight_dev, double scale, float *x_dev)
{
    if (!s || !U_dev || !E_dev || !chi_tight_dev || !x_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (!(scale > 0.0)) return fail(VESIS_E_ARG, "scale must be > 0");
    launch_features(U_dev, E_dev, s->G, chi_tight_dev, (float)s->cfa, (float)scale, x_dev, s->st);
    VTRY(last_launch("features"));
    VCK(cudaStreamSynchronize(s->st));
    return VESIS_OK;
}

int vesis_atom_forces(vesis_system s, const uint8_t *chi_dev, const double *xyz,
                      const float *E_dev, double *grad_out, double *energy_out)
{
    if (!s || !chi_dev || !grad_out) return fail(VESIS_E_ARG, "NULL argument");
    if (xyz) VTRY(vesis_set_positions(s, xyz));
    else enq_pack(s, s->d_xyz);
    double *bk = bank(s, 0);
    const float *E = E_dev;
    if (!E || energy_out) {
        enq_fields(s, s->d_U[0], s->d_E[0], bk);
        E = s->d_E[0];
    } else {
        enq_far(s, bk);
    }
    enq_gradient(s, chi_dev, E, s->d_xyz, bk);
    if (energy_out) {
        enq_terms(s, chi_dev, s->d_U[0], s->d_E[0], bk);
        VTRY(last_launch("atom_forces"));
        VTRY(read_bank(s, bk));
        *energy_out = s->h_scal[S_TOTAL];
    }
    VTRY(last_launch("atom_forces"));
    VCK(cudaMemcpyAsync(grad_out, s->d_grad, 3 * sizeof(double) * s->n,
                        cudaMemcpyDeviceToHost, s->st));
    VCK(cudaStreamSynchronize(s->st));
    for (int i = 0; i < 3 * s->n; ++i)
        if (!std::isfinite(grad_out[i])) return fail(VESIS_E_NAN, "non-finite gradient");
    return VESIS_OK;
}

int vesis_relax(vesis_system s, uint8_t *chi_dev, double *xyz_inout,
                const vesis_relax_opts *opts_in, vesis_relax_stats *stats_out)
{
    if (!s || !chi_dev || !xyz_inout) return fail(VESIS_E_ARG, "NULL argument");
    vesis_relax_opts o;
    if (opts_in) o = *opts_in;
    else vesis_default_relax_opts(&o);
    if (o.max_outer < 0 || o.window < 1 || o.max_flip_rounds < 1 ||
        o.max_gd_retries < 0 || !(o.alpha > 0.0 && o.alpha < 1.0) || !(o.M0 > 0.0) ||
        (o.resume != 0 && o.resume != 1))
        return fail(VESIS_E_ARG, "invalid relax options");
    if (o.resume && !s->rstate.valid)
        return fail(VESIS_E_ARG, "no relaxation state to resume");
    const vesis_relax_state from = s->rstate;
    s->rstate.valid = 0;     // written again when this call ends normally
    vesis_relax_stats st;
    std::memset(&st, 0, sizeof(st));
    const long long GN = s->G * (long long)s->n;
    const long long FN = (long long)s->nfar * s->n;
    const long long NN = (long long)s->n * s->n;

    VTRY(vesis_set_positions(s, xyz_inout));
    int cur = 0, trial = 1;
    enq_fields(s, s->d_U[cur], s->d_E[cur], bank(s, cur));
    enq_ss(s, s->d_xyz, bank(s, cur));
    enq_terms(s, chi_dev, s->d_U[cur], s->d_E[cur], bank(s, cur));
    // from here on d_W is the exact convolution of chi_dev: only the sweep
    // changes the labels in this call, and it keeps d_W current
    count_launch();
    k_gd_init<<<1, 1, 0, s->st>>>(s->d_gd, o.resume ? from.M : o.M0, o.resume ? from.ncnt : 0);
    VTRY(last_launch("relax init"));
    VTRY(read_bank(s, bank(s, cur)));
    st.pair_evals += GN + FN + NN;
    double G_prev = o.resume ? from.G_prev : s->h_scal[S_TOTAL];
    if (!std::isfinite(s->h_scal[S_TOTAL]))
        return fail(VESIS_E_NAN, "non-finite initial energy");

    int k = o.resume ? from.k : 0, stable = o.resume ? from.stable : 0;
    int reason = 2, status = VESIS_OK;
    double gmax = 0.0;
    // One outer iteration waits on the host once: the sweep, the gradient
    // and the first trial step are enqueued together, and their records
    // come back with one synchronisation (a rejected trial costs one more).
    auto enq_trial = [&]() {
        launch_mobility(s->d_xyz, s->d_grad, s->d_gmax, &s->d_gd->M, s->d_xyz_new, 3 * s->n,
                        s->st);
        enq_pack(s, s->d_xyz_new);
        enq_fields(s, s->d_U[trial], s->d_E[trial], bank(s, trial));
        enq_ss(s, s->d_xyz_new, bank(s, trial));
        enq_terms(s, chi_dev, s->d_U[trial], s->d_E[trial], bank(s, trial), true);
        count_launch();
        k_gd_decide<<<1, 1, 0, s->st>>>(s->d_gd, bank(s, cur), bank(s, trial), s->d_oob,
                                        o.ncnt_star, o.dgstar_frac, o.alpha, s->d_gmax,
                                        o.tol_grad);
    };
    auto copy_trial = [&]() -> int {
        VCK(cudaMemcpyAsync(s->h_gd, s->d_gd, sizeof(GdState), cudaMemcpyDeviceToHost, s->st));
        VCK(cudaMemcpyAsync(s->h_scal2, bank(s, trial), S_BANK * sizeof(double),
                            cudaMemcpyDeviceToHost, s->st));
        return VESIS_OK;
    };
    while (k < o.max_outer) {
        RoundState rs;
        int sweep_sp = -2;
        {
            NvtxRange range("vesis: flip sweep");
            VTRY(run_blsm(s, chi_dev, s->d_U[cur], o.max_flip_rounds, &rs, true, &sweep_sp));
        }
        // Step 3.1-3.2: gradient and G_old at (Gamma^{k+1}, R^k); the
        // solute-solute terms at R^k are current (the start or the accepted
        // trial evaluated them last)
        {
            NvtxRange range("vesis: gradient");
            enq_gradient(s, chi_dev, s->d_E[cur], s->d_xyz, bank(s, cur), true);
            enq_terms(s, chi_dev, s->d_U[cur], s->d_E[cur], bank(s, cur), true);
        }
        // Step 3.3-3.4: the first trial step, enqueued before the gradient
        // test is known here (void if that test ends the relaxation)
        int retries = 0;
        bool accepted = false;
        double G_new = 0.0;
        {
            NvtxRange range("vesis: trial steps");
            enq_trial();
            VTRY(last_launch("relax iteration"));
            VCK(cudaMemcpyAsync(s->h_u64, s->d_gmax, sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, s->st));
            VCK(cudaMemcpyAsync(s->h_scal, bank(s, cur), S_BANK * sizeof(double),
                                cudaMemcpyDeviceToHost, s->st));
            VTRY(copy_trial());
            VCK(cudaStreamSynchronize(s->st));
        }
        if (sweep_sp != -2) VTRY(finish_blsm(s, sweep_sp, &rs));
        st.flip_rounds += rs.round;
        st.flips += (long long)rs.total_flips;
        const double G_old = s->h_scal[S_TOTAL];
        std::memcpy(&gmax, s->h_u64, sizeof(double));
        st.pair_evals += (s->G - (long long)s->h_scal[S_NSOL]) * s->n + FN;
        if (!std::isfinite(gmax) || gmax >= 1.0e308) {
            enq_pack(s, s->d_xyz);   // the void trial moved the packed atoms
            status = fail(VESIS_E_NAN, "non-finite gradient");
            break;
        }
        if (gmax < o.tol_grad) {
            enq_pack(s, s->d_xyz);
            reason = 0;
            break;
        }
        {
            NvtxRange range("vesis: trial steps");
            for (;;) {
                st.gd_trials += 1;
                st.pair_evals += GN + FN + NN;
                if (s->h_gd->decision == 0) {
                    accepted = true;
                    G_new = s->h_scal2[S_TOTAL];
                    break;
                }
                if (++retries > o.max_gd_retries) break;
                enq_trial();
                VTRY(last_launch("relax trial"));
                VTRY(copy_trial());
                VCK(cudaStreamSynchronize(s->st));
            }
        }
        if (!accepted) {
            enq_pack(s, s->d_xyz);   // keep the packed atoms on R^k
            reason = 3;
            status = VESIS_W_NOT_CONVERGED;
            break;
        }
        std::swap(cur, trial);
        std::swap(s->d_xyz, s->d_xyz_new);
        ++k;
        if (s->hist && st.records < s->hist_cap) {
            vesis_iter_record &rec = s->hist[st.records++];
            rec.k = k;
            rec.rounds = rs.round;
            rec.flips = (long long)rs.total_flips;
            rec.trials = retries + 1;
            rec.ncnt = s->h_gd->ncnt;
            rec.G = G_new;
            rec.G_old = G_old;
            rec.M = s->h_gd->M;
            rec.max_grad = gmax;
        }
        // Steps 4-5: energy change between consecutive accepted iterates
        const double d_abs = std::fabs(G_new - G_prev);
        const double d_rel = G_new != 0.0 ? d_abs / std::fabs(G_new) : INFINITY;
        G_prev = G_new;
        if (d_abs < o.tol_energy || d_rel < o.tol_energy) {
            if (++stable >= o.window) {
                reason = 1;
                break;
            }
        } else {
            stable = 0;
        }
    }
    if (status == VESIS_OK && reason == 2) status = VESIS_W_NOT_CONVERGED;
    // final state: bank(cur) already holds every term at (chi, R^k) - the
    // start, the gradient step after the last sweep or the accepted trial
    // wrote it last - so it is only read back
    if (status >= 0) {
        VTRY(last_launch("relax final"));
        VTRY(read_bank(s, bank(s, cur)));
        fill_terms(s->h_scal, true, st.terms);
        st.G = st.terms[5];
        VCK(cudaMemcpyAsync(s->h_gd, s->d_gd, sizeof(GdState),
                            cudaMemcpyDeviceToHost, s->st));
        VCK(cudaMemcpyAsync(xyz_inout, s->d_xyz, 3 * sizeof(double) * s->n,
                            cudaMemcpyDeviceToHost, s->st));
        VCK(cudaStreamSynchronize(s->st));
        st.M = s->h_gd->M;
        s->rstate.k = k;
        s->rstate.ncnt = s->h_gd->ncnt;
        s->rstate.stable = stable;
        s->rstate.M = s->h_gd->M;
        s->rstate.G_prev = G_prev;
        s->rstate.valid = 1;
    }
    st.status = status;
    st.iterations = k;
    st.stop_reason = reason;
    st.max_grad = gmax;
    if (stats_out) *stats_out = st;
    return status;
}

int vesis_set_history(vesis_system s, vesis_iter_record *records, int capacity)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    if (capacity < 0) return fail(VESIS_E_ARG, "capacity must be >= 0");
    s->hist = capacity > 0 ? records : nullptr;
    s->hist_cap = records ? capacity : 0;
    return VESIS_OK;
}

int vesis_get_state(vesis_system s, vesis_relax_state *out)
{
    if (!s || !out) return fail(VESIS_E_ARG, "NULL argument");
    *out = s->rstate;
    return VESIS_OK;
}

int vesis_set_state(vesis_system s, const vesis_relax_state *in)
{
    if (!s || !in) return fail(VESIS_E_ARG, "NULL argument");
    if (in->k < 0 || in->ncnt < 0 || in->stable < 0 || !(in->M > 0.0) ||
        !std::isfinite(in->M) || !std::isfinite(in->G_prev) ||
        (in->valid != 0 && in->valid != 1))
        return fail(VESIS_E_ARG, "invalid relaxation state");
    s->rstate = *in;
    return VESIS_OK;
}

int vesis_set_wait_limit(vesis_system s, long long polls)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    if (polls < 0) return fail(VESIS_E_ARG, "polls must be >= 0");
    s->spin_limit = polls;
    return VESIS_OK;
}

int vesis_set_sweep_stamps(vesis_system s, int mode)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    if (mode < -1 || mode > 1) return fail(VESIS_E_ARG, "mode must be -1, 0 or 1");
    s->sweep_stamps = mode;
    return VESIS_OK;
}

int vesis_set_tiles(vesis_system s, int energy_pencil, int force_atoms)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    if (energy_pencil != 4 && energy_pencil != 8 && energy_pencil != 16)
        return fail(VESIS_E_ARG, "energy_pencil must be 4, 8 or 16");
    if (force_atoms != 2 && force_atoms != 4)
        return fail(VESIS_E_ARG, "force_atoms must be 2 or 4");
    VCK(cudaStreamSynchronize(s->st));
    s->pe_pts = energy_pencil;
    const ForcePlan fp = plan_pair_force(s->G, s->n, s->nsm, force_atoms);
    // the partial buffer was sized for this chunk count at set-up
    if (fp.nchunk != s->fplan.nchunk) return fail(VESIS_E_CUDA, "gradient chunk plan changed");
    s->fplan = fp;
    return VESIS_OK;
}

int vesis_get_tiles(vesis_system s, int *energy_pencil, int *force_atoms)
{
    if (!s) return fail(VESIS_E_ARG, "NULL system");
    if (energy_pencil) *energy_pencil = s->pe_pts;
    if (force_atoms) *force_atoms = s->fplan.apt;
    return VESIS_OK;
}

int vesis_autotune(vesis_system s, const uint8_t *chi_dev, int reps, double *times_ms_out)
{
    if (!s || !chi_dev) return fail(VESIS_E_ARG, "NULL argument");
    if (reps < 1 || reps > 1000) return fail(VESIS_E_ARG, "reps must be in 1..1000");
    static const int kPencil[3] = {4, 8, 16}, kAtoms[2] = {2, 4};
    double ms[5] = {0, 0, 0, 0, 0};
    // the trial buffers are scratch between calls; the count of solvent
    // cells the gradient kernel keeps for the timing report is put back
    float *U = s->d_U[1], *E = s->d_E[1];
    VCK(cudaMemcpyAsync(s->h_u64, s->d_fcount, sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s->st));
    VCK(cudaStreamSynchronize(s->st));
    const unsigned long long fcount = *s->h_u64;
    struct Events {
        vesis_system s;
        cudaEvent_t a, b;
        ~Events()
        {
            s->ev_pool.push_back(a);
            s->ev_pool.push_back(b);
        }
    } ev{s, take_event(s), take_event(s)};
    cudaEvent_t a = ev.a, b = ev.b;
    auto timed = [&](auto &&launch, double *out) -> int {
        launch();   // warm-up
        VCK(cudaEventRecord(a, s->st));
        for (int i = 0; i < reps; ++i) launch();
        VCK(cudaEventRecord(b, s->st));
        VCK(cudaEventSynchronize(b));
        float t = 0.f;
        VCK(cudaEventElapsedTime(&t, a, b));
        *out = (double)t / reps;
        return VESIS_OK;
    };
    for (int v = 0; v < 3; ++v) {
        const int P = kPencil[v];
        VTRY(timed([&] {
            launch_pair_energy_grid(s->g, atoms_view(s), (float)s->p.rho_w, (float)s->cfa,
                                    s->rmin2, U, E, E + s->G, E + 2 * s->G, P, s->st);
        }, &ms[v]));
    }
    for (int v = 0; v < 2; ++v) {
        const ForcePlan fp = plan_pair_force(s->G, s->n, s->nsm, kAtoms[v]);
        VTRY(timed([&] {
            launch_pair_force_grid(s->g, fp, chi_dev, E, E + s->G, E + 2 * s->G,
                                   atoms_view(s), s->rmin2, s->d_fpart, s->d_fcount, s->st);
        }, &ms[3 + v]));
    }
    VTRY(last_launch("autotune"));
    *s->h_u64 = fcount;
    VCK(cudaMemcpyAsync(s->d_fcount, s->h_u64, sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, s->st));
    if (times_ms_out) std::memcpy(times_ms_out, ms, sizeof(ms));
    int best = 1;
    for (int v = 0; v < 3; ++v)
        if (ms[v] < ms[best]) best = v;
    return vesis_set_tiles(s, kPencil[best], ms[3] < ms[4] ? 2 : 4);
}

int vesis_relax_batch(int nsys, vesis_system *systems, uint8_t *const *chi_dev,
                      double *const *xyz_inout, const vesis_relax_opts *opts,
                      int threads, int sweep_slots, vesis_relax_stats *stats_out,
                      int *status_out)
{
    if (nsys < 0) return fail(VESIS_E_ARG, "nsys must be >= 0");
    if (nsys == 0) return VESIS_OK;
    if (!systems || !chi_dev || !xyz_inout) return fail(VESIS_E_ARG, "NULL argument");
    if (threads < 1 || threads > 256) return fail(VESIS_E_ARG, "threads must be in 1..256");
    if (sweep_slots < 1 || sweep_slots > 16)
        return fail(VESIS_E_ARG, "sweep_slots must be in 1..16");
    int dev = -1;
    for (int i = 0; i < nsys; ++i) {
        if (!systems[i] || !chi_dev[i] || !xyz_inout[i])
            return fail(VESIS_E_ARG, "NULL system or buffer at index " + std::to_string(i));
        for (int j = 0; j < i; ++j)
            if (systems[j] == systems[i])
                return fail(VESIS_E_ARG, "a system appears twice in the batch");
        if (dev < 0) dev = systems[i]->dev;
        if (systems[i]->dev != dev) return fail(VESIS_E_ARG, "systems are on different devices");
    }
    int dev0 = 0;
    VCK(cudaGetDevice(&dev0));
    VCK(cudaSetDevice(dev));
    // one wave of sweep blocks shared by the admitted sweeps
    SweepGate gate;
    int wave = systems[0]->sweep_blocks;
    for (int i = 1; i < nsys; ++i) wave = std::min(wave, systems[i]->sweep_blocks);
    gate.free_slots = std::min(sweep_slots, std::max(1, wave));
    gate.blocks = std::max(1, wave / gate.free_slots);
    // every system runs on a private non-blocking stream for the call; the
    // caller's streams are drained first and handed back afterwards
    std::vector<cudaStream_t> own(nsys, nullptr), prev(nsys, nullptr);
    int rc = VESIS_OK;
    for (int i = 0; i < nsys && rc == VESIS_OK; ++i) {
        if (cudaStreamSynchronize(systems[i]->st) != cudaSuccess ||
            cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking) != cudaSuccess)
            rc = fail(VESIS_E_CUDA, "batch stream set-up failed");
    }
    std::vector<int> status(nsys, VESIS_E_CUDA);
    std::vector<std::string> msg(nsys);
    if (rc == VESIS_OK) {
        for (int i = 0; i < nsys; ++i) {
            prev[i] = systems[i]->st;
            systems[i]->st = own[i];
            systems[i]->gate = &gate;
        }
        // largest systems first (longest-processing-time order)
        std::vector<int> order(nsys);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return systems[x]->G * (long long)systems[x]->n >
                   systems[y]->G * (long long)systems[y]->n;
        });
        std::atomic<int> next{0};
        auto worker = [&] {
            cudaSetDevice(dev);
            for (;;) {
                const int q = next.fetch_add(1);
                if (q >= nsys) break;
                const int i = order[q];
                vesis_relax_stats st;
                std::memset(&st, 0, sizeof(st));
                status[i] = vesis_relax(systems[i], chi_dev[i], xyz_inout[i], opts, &st);
                if (status[i] < 0) msg[i] = g_err;
                if (stats_out) stats_out[i] = st;
            }
        };
        const int nt = std::min(threads, nsys);
        std::vector<std::thread> pool;
        try {
            pool.reserve(nt);
            for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
        } catch (...) {
            // no more threads: the ones that started drain the queue
        }
        if (pool.empty()) worker();
        for (auto &t : pool) t.join();
        for (int i = 0; i < nsys; ++i) {
            cudaStreamSynchronize(own[i]);
            systems[i]->st = prev[i];
            systems[i]->gate = nullptr;
        }
        for (int i = 0; i < nsys && rc == VESIS_OK; ++i)
            if (status[i] < 0) rc = fail(status[i], "system " + std::to_string(i) + ": " + msg[i]);
    }
    for (int i = 0; i < nsys; ++i)
        if (own[i]) cudaStreamDestroy(own[i]);
    if (status_out) std::memcpy(status_out, status.data(), nsys * sizeof(int));
    cudaSetDevice(dev0);
    return rc;
}

}  // extern "C"
