// Persistent narrow-band flip sweep (Sec. 3.1, Step 2) for sm_103a.
//
// All flip rounds of one interface relaxation run in a single cooperative
// launch.  The grid is cut into 8^3 tiles; only tiles holding candidate
// cells (a face neighbour with the other label) are active, which is the
// band around the interface the paper restricts the flips to.  Per round:
//
//   phase A (active tiles): dE = c [s (1 - 2w) - g0] - s h^3 U in FP64 for
//     candidates (Eq. dGj1/dGj2); a cell with dE < 0 gets the 32-bit key
//     bits(float(dE)) (the raw bits of a negative float grow as the value
//     falls), every other cell the key 0.  A tile without candidates turns
//     inactive.
//   barrier
//   phase B (tiles with a negative candidate): the keys of the tile and a
//     halo of r cells arrive in shared memory by one TMA box load (cells
//     outside the grid read 0 = no key); the window maximum over the cube of
//     half-width r comes from three separable passes; a cell is selected when
//     its key is that maximum and no other cell of its window holds the same
//     key at a smaller linear index.  This is the order (float(dE), index)
//     of the serial min-heap, restricted to one winner per window.  Selected
//     cells flip; +-q_a q_b q_c is added to W over each flipped cell's window
//     with integer atomics, so W stays the exact convolution; the tiles of
//     the flipped cells and of their face neighbours are activated.
//   barrier; stop when the round flipped nothing.
//
// Selected cells are more than r apart, so they do not interact through the
// kernel and a round lowers the energy by exactly the sum of their dE.
// Every spin (grid barrier, TMA completion) is bounded: on timeout an error
// flag is raised, in-flight copies are awaited (again bounded) and every
// block returns.
#include <cuda.h>

#include <cstring>

#include "vesis_internal.cuh"

namespace vesis {

constexpr int TS = 8;             // tile edge
constexpr int TC = TS * TS * TS;  // cells per tile
constexpr int SW_THREADS = 256;
constexpr int BXW = TS + 16;      // key box width along z (start k0 - 8)
constexpr long long kSpinLimit = 1ll << 26;
constexpr long long kMbarSpin = 1ll << 24;
constexpr int kMaxWinners = TC;   // every cell of a tile may tie

struct SweepArgs {
    GridDesc g;
    KernelW kw;
    FlipConst fc;
    uint8_t *chi;
    uint32_t *W;
    const float *U;
    uint32_t *K;        // 32-bit keys
    double *dE;
    uint8_t *act0, *act1, *tneg;
    int ntx, nty, ntz;
    unsigned *cnt;      // [3] flips per round, cycled
    unsigned *bar;      // [2] arrival count, generation
    int *err;
    unsigned long long *part_flips;   // [gridDim.x]
    double *part_dE;                  // [gridDim.x]
    int *rounds_out;
    int *capped_out;
    int max_rounds;
    int use_tma;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool grid_barrier(const SweepArgs &A)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = A.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(A.bar, 1u);
        if (arrived == gridDim.x - 1) {
            A.bar[0] = 0;
            __threadfence();
            atomicAdd(A.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                if (++spins > kSpinLimit || *(volatile int *)A.err) {
                    atomicExch(A.err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)A.err == 0;
}

// Bounded wait for the phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ double flip_dE_s(uint8_t chi_j, unsigned W, float U,
                                            const FlipConst &fc)
{
    const double w = __dmul_rn((double)W, fc.invD3);
    const double s = chi_j ? -1.0 : 1.0;
    const double a = __dsub_rn(__dmul_rn(s, __dsub_rn(1.0, __dmul_rn(2.0, w))), fc.g0);
    const double t1 = __dmul_rn(fc.c, a);
    const double t2 = __dmul_rn(fc.h3, (double)U);
    return __dsub_rn(t1, __dmul_rn(s, t2));
}

__device__ __forceinline__ void tile_origin(const SweepArgs &A, int t, int &i0,
                                            int &j0, int &k0)
{
    const int tk = t % A.ntz;
    const int tj = (t / A.ntz) % A.nty;
    const int ti = t / (A.ntz * A.nty);
    i0 = ti * TS;
    j0 = tj * TS;
    k0 = tk * TS;
}

__device__ __forceinline__ void mark_tile(const SweepArgs &A, uint8_t *act,
                                          int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= A.g.nx || j >= A.g.ny || k >= A.g.nz) return;
    act[((i / TS) * A.nty + (j / TS)) * A.ntz + (k / TS)] = 1;
}

struct SweepShared {
    uint8_t chi[(TS + 2) * (TS + 2) * (TS + 2)];
    int list[SW_THREADS];
    int wc[SW_THREADS / 32];
    int nlist;
    long long win_p[kMaxWinners];
    uint32_t win_key[kMaxWinners];
    int win_pos[kMaxWinners];
    int win_ok[kMaxWinners];
    double e[SW_THREADS / 32];
    unsigned long long mbar;
};

// Labels, W and keys change under other blocks between rounds: every read
// of them goes to L2 (ld.global.cg) so no stale L1 line is used.

// Phase A for one tile: keys and flip energies of its cells.
__device__ void phase_keys(const SweepArgs &A, SweepShared &S, int t,
                           uint8_t *act_next)
{
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    constexpr int E = TS + 2;
    for (int idx = threadIdx.x; idx < E * E * E; idx += SW_THREADS) {
        const int hz = idx % E, hy = (idx / E) % E, hx = idx / (E * E);
        const int i = i0 - 1 + hx, j = j0 - 1 + hy, k = k0 - 1 + hz;
        uint8_t v = 0;
        if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz)
            v = __ldcg(A.chi + (long long)i * nyz + (long long)j * g.nz + k);
        S.chi[idx] = v;
    }
    __syncthreads();
    bool cand_any = false, neg_any = false;
#pragma unroll
    for (int u = 0; u < TC / SW_THREADS; ++u) {
        const int c = threadIdx.x + u * SW_THREADS;
        const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
        const int i = i0 + x, j = j0 + y, k = k0 + z;
        if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
        const int h = ((x + 1) * E + (y + 1)) * E + (z + 1);
        const uint8_t v = S.chi[h];
        const bool cand = (S.chi[h - E * E] != v) | (S.chi[h + E * E] != v) |
                          (S.chi[h - E] != v) | (S.chi[h + E] != v) |
                          (S.chi[h - 1] != v) | (S.chi[h + 1] != v);
        const long long p = (long long)i * nyz + (long long)j * g.nz + k;
        uint32_t key = 0;
        if (cand) {
            cand_any = true;
            const double e = flip_dE_s(v, __ldcg(A.W + p), __ldg(A.U + p), A.fc);
            if (e < 0.0) {
                A.dE[p] = e;
                key = __float_as_uint(__double2float_rn(e));
                neg_any = true;
            }
        }
        A.K[p] = key;
    }
    const int ca = __syncthreads_or(cand_any);
    const int na = __syncthreads_or(neg_any);
    if (threadIdx.x == 0) {
        act_next[t] = (uint8_t)(ca != 0);
        A.tneg[t] = (uint8_t)(na != 0);
    }
}

// Phase B for one tile: window maximum, ties, flips, W update, activation.
__device__ bool phase_flip(const CUtensorMap *tmap, const SweepArgs &A,
                           SweepShared &S, uint32_t *Kh, uint32_t &mbar_phase,
                           int t, uint8_t *act_next, unsigned &nflip, double &esum)
{
    const int r = A.kw.r;
    const int BY = TS + 2 * r;     // box extent along y and x (i)
    const int w = 2 * r + 1;
    uint32_t *M1 = Kh + BY * BY * BXW;          // [BY][BY][TS]
    uint32_t *M2 = M1 + BY * BY * TS;           // [BY][TS][TS]
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    if (A.use_tma) {
        if (threadIdx.x == 0) {
            const uint32_t bar = smem_addr(&S.mbar);
            const uint32_t bytes = (uint32_t)(BXW * BY * BY * 4);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(bar), "r"(bytes) : "memory");
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4}], [%5];"
                :: "r"(smem_addr(Kh)), "l"(reinterpret_cast<uint64_t>(tmap)),
                   "r"(k0 - 8), "r"(j0 - r), "r"(i0 - r), "r"(bar)
                : "memory");
        }
        const bool ok = mbar_wait(smem_addr(&S.mbar), mbar_phase, kMbarSpin);
        if (!ok) {
            atomicExch(A.err, 1);
            mbar_wait(smem_addr(&S.mbar), mbar_phase, kMbarSpin);
            return false;
        }
        mbar_phase ^= 1u;
    } else {
        for (int idx = threadIdx.x; idx < BY * BY * BXW; idx += SW_THREADS) {
            const int hz = idx % BXW, hy = (idx / BXW) % BY, hx = idx / (BXW * BY);
            const int i = i0 - r + hx, j = j0 - r + hy, k = k0 - 8 + hz;
            uint32_t v = 0;
            if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz)
                v = __ldcg(A.K + (long long)i * nyz + (long long)j * g.nz + k);
            Kh[idx] = v;
        }
    }
    __syncthreads();
    // z pass: tile cell z sits at box column 8 + z
    for (int idx = threadIdx.x; idx < BY * BY * TS; idx += SW_THREADS) {
        const int z = idx % TS, hy = (idx / TS) % BY, hx = idx / (TS * BY);
        const uint32_t *col = Kh + (hx * BY + hy) * BXW + (8 + z - r);
        uint32_t m = col[0];
        for (int d = 1; d < w; ++d) m = max(m, col[d]);
        M1[idx] = m;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < BY * TS * TS; idx += SW_THREADS) {
        const int z = idx % TS, y = (idx / TS) % TS, hx = idx / (TS * TS);
        const uint32_t *col = M1 + (hx * BY + y) * TS + z;
        uint32_t m = col[0];
        for (int d = 1; d < w; ++d) m = max(m, col[d * TS]);
        M2[idx] = m;
    }
    __syncthreads();
    // window maxima; the winners are listed in increasing cell order
    // (ballot compaction), so everything after is independent of timing
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    int nw = 0;
#pragma unroll
    for (int u = 0; u < TC / SW_THREADS; ++u) {
        const int c = threadIdx.x + u * SW_THREADS;
        const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
        const int pos = ((x + r) * BY + (y + r)) * BXW + (8 + z);
        const uint32_t key = Kh[pos];
        bool win = false;
        if (key != 0u) {
            const uint32_t *col = M2 + (x * TS + y) * TS + z;
            uint32_t m = col[0];
            for (int d = 1; d < w; ++d) m = max(m, col[d * TS * TS]);
            win = (m == key);
        }
        const unsigned b = __ballot_sync(0xffffffffu, win);
        if (lane == 0) S.wc[wp] = __popc(b);
        __syncthreads();
        int off = nw, tot = 0;
#pragma unroll
        for (int q = 0; q < SW_THREADS / 32; ++q) {
            if (q < wp) off += S.wc[q];
            tot += S.wc[q];
        }
        if (win) {
            const int slot = off + __popc(b & ((1u << lane) - 1u));
            S.win_p[slot] = (long long)(i0 + x) * nyz + (long long)(j0 + y) * g.nz + (k0 + z);
            S.win_key[slot] = key;
            S.win_pos[slot] = pos;
            S.win_ok[slot] = 1;
        }
        nw += tot;
        __syncthreads();
    }
    // ties: an equal key at a smaller index inside the window loses the
    // winner its place (box order (x, y, z) is the linear index order)
    for (int q = 0; q < nw; ++q) {
        const int pos = S.win_pos[q];
        const uint32_t key = S.win_key[q];
        const int cz = pos % BXW, cy = (pos / BXW) % BY, cx = pos / (BXW * BY);
        bool lose = false;
        for (int idx = threadIdx.x; idx < w * w * w; idx += SW_THREADS) {
            const int dz = idx % w - r, dy = (idx / w) % w - r, dx = idx / (w * w) - r;
            const int qp = ((cx + dx) * BY + (cy + dy)) * BXW + (cz + dz);
            if (qp < pos && Kh[qp] == key) lose = true;
        }
        if (__syncthreads_or(lose) && threadIdx.x == 0) S.win_ok[q] = 0;
    }
    __syncthreads();
    // flips and the exact energy change of this tile (fixed order)
    if (threadIdx.x == 0) {
        double te = 0.0;
        unsigned nf = 0;
        for (int q = 0; q < nw; ++q) {
            if (!S.win_ok[q]) continue;
            const long long p = S.win_p[q];
            A.chi[p] = (uint8_t)(1 - __ldcg(A.chi + p));
            te += __ldcg(A.dE + p);
            ++nf;
        }
        esum += te;
        nflip += nf;
    }
    __syncthreads();
    for (int q = 0; q < nw; ++q) {
        if (!S.win_ok[q]) continue;
        const long long p = S.win_p[q];
        const int i = (int)(p / nyz), j = (int)((p / g.nz) % g.ny), k = (int)(p % g.nz);
        const int sgn = __ldcg(A.chi + p) ? 1 : -1;   // already flipped
        for (int idx = threadIdx.x; idx < w * w * w; idx += SW_THREADS) {
            const int c = idx % w, b = (idx / w) % w, a = idx / (w * w);
            const int ii = i + a - r, jj = j + b - r, kk = k + c - r;
            if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
            const int val = A.kw.q[a] * A.kw.q[b] * A.kw.q[c];
            atomicAdd(&A.W[(long long)ii * nyz + (long long)jj * g.nz + kk],
                      (unsigned)(sgn * val));
        }
        if (threadIdx.x < 7) {
            const int d = threadIdx.x;
            const int di = (d == 1) - (d == 2), dj = (d == 3) - (d == 4),
                      dk = (d == 5) - (d == 6);
            mark_tile(A, act_next, i + di, j + dj, k + dk);
        }
    }
    __syncthreads();
    return true;
}

// Collects, in increasing order, this block's tiles t = blockIdx.x + k *
// gridDim.x (k in [base, base + SW_THREADS)) whose flag is set; returns
// the count (list in S.list).  With `clear`, unflagged tiles get nxt = 0
// and tneg = 0.
__device__ int gather_tiles(const SweepArgs &A, SweepShared &S, const uint8_t *flags,
                            int base, int ntiles, uint8_t *clear_nxt)
{
    const int k = base + threadIdx.x;
    const long long t = (long long)blockIdx.x + (long long)k * gridDim.x;
    bool fl = false;
    if (t < ntiles) {
        fl = __ldcg(flags + t) != 0;
        if (!fl && clear_nxt) {
            clear_nxt[t] = 0;
            A.tneg[t] = 0;
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, fl);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) S.wc[wp] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < SW_THREADS / 32; ++q) {
        if (q < wp) off += S.wc[q];
        tot += S.wc[q];
    }
    if (fl) S.list[off + __popc(b & ((1u << lane) - 1u))] = (int)t;
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(SW_THREADS)
k_sweep(const __grid_constant__ CUtensorMap tmap, SweepArgs A)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ SweepShared S;
    uint32_t *Kh = reinterpret_cast<uint32_t *>(dsm);
    const int ntiles = A.ntx * A.nty * A.ntz;
    const int per_block = (ntiles + gridDim.x - 1) / gridDim.x;
    uint32_t mbar_phase = 0;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;"
                     :: "r"(smem_addr(&S.mbar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned nflip = 0;       // thread 0 only
    double esum = 0.0;        // thread 0 only
    int round = 0, capped = 0;
    for (;;) {
        uint8_t *cur = (round & 1) ? A.act1 : A.act0;
        uint8_t *nxt = (round & 1) ? A.act0 : A.act1;
        if (blockIdx.x == 0 && threadIdx.x == 0) A.cnt[(round + 1) % 3] = 0;
        for (int base = 0; base < per_block; base += SW_THREADS) {
            const int n = gather_tiles(A, S, cur, base, ntiles, nxt);
            for (int q = 0; q < n; ++q) phase_keys(A, S, S.list[q], nxt);
            __syncthreads();
        }
        if (!grid_barrier(A)) return;
        const unsigned before = nflip;
        for (int base = 0; base < per_block; base += SW_THREADS) {
            const int n = gather_tiles(A, S, A.tneg, base, ntiles, nullptr);
            for (int q = 0; q < n; ++q)
                if (!phase_flip(&tmap, A, S, Kh, mbar_phase, S.list[q], nxt, nflip, esum))
                    return;
            __syncthreads();
        }
        if (threadIdx.x == 0 && nflip != before) atomicAdd(&A.cnt[round % 3], nflip - before);
        if (!grid_barrier(A)) return;
        const unsigned n = *(volatile unsigned *)&A.cnt[round % 3];
        if (n == 0) break;
        ++round;
        if (round >= A.max_rounds) {
            capped = 1;
            break;
        }
    }
    if (threadIdx.x == 0) {
        A.part_flips[blockIdx.x] = nflip;
        A.part_dE[blockIdx.x] = esum;
        if (blockIdx.x == 0) {
            *A.rounds_out = round;
            *A.capped_out = capped;
        }
    }
}

__global__ void k_sweep_final(const unsigned long long *part_flips,
                              const double *part_dE, int nb, const int *rounds,
                              const int *capped, RoundState *rs)
{
    unsigned long long f = 0;
    double e = 0.0;
    for (int b = 0; b < nb; ++b) {
        f += part_flips[b];
        e += part_dE[b];
    }
    rs->done = 1;
    rs->round = *rounds;
    rs->capped = *capped;
    rs->round_flips = 0;
    rs->total_flips = f;
    rs->round_dE = 0.0;
    rs->total_dE = e;
}

size_t sweep_smem_bytes(int r)
{
    const size_t BY = TS + 2 * r;
    return sizeof(uint32_t) * (BY * BY * BXW + BY * BY * TS + BY * TS * TS);
}

int sweep_tiles(const GridDesc &g)
{
    return ((g.nx + TS - 1) / TS) * ((g.ny + TS - 1) / TS) * ((g.nz + TS - 1) / TS);
}

cudaError_t sweep_grid_size(int r, int nsm, int *blocks)
{
    const size_t sm = sweep_smem_bytes(r);
    cudaError_t e = cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    int per = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep, SW_THREADS, sm);
    if (e != cudaSuccess) return e;
    per = per > 4 ? 4 : per;
    *blocks = per * nsm;
    return *blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// TMA descriptor of the key volume: dims (nz, ny, nx) of uint32, box
// (TS + 16, TS + 2r, TS + 2r); zero fill outside.  Needs nz % 4 == 0 (row
// pitch a multiple of 16 bytes).
bool sweep_make_tmap(const GridDesc &g, int r, uint32_t *K, void *tmap_out)
{
    if (g.nz % 4 != 0) return false;
    typedef CUresult (*encode_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *,
                                 const cuuint32_t *, const cuuint32_t *,
                                 CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nz, (cuuint64_t)g.ny, (cuuint64_t)g.nx};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nz * 4, (cuuint64_t)g.nz * g.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)BXW, (cuuint32_t)(TS + 2 * r),
                               (cuuint32_t)(TS + 2 * r)};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult res = ((encode_t)fn)(
        reinterpret_cast<CUtensorMap *>(tmap_out), CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, K,
        dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return res == CUDA_SUCCESS;
}

size_t sweep_tmap_bytes() { return sizeof(CUtensorMap); }

cudaError_t launch_sweep(const void *tmap, int use_tma, const GridDesc &g,
                         const KernelW &kw, const FlipConst &fc, uint8_t *chi,
                         uint32_t *W, const float *U, uint32_t *K, double *dE,
                         uint8_t *act, uint8_t *tneg, unsigned *ctl, int *err,
                         unsigned long long *part_flips, double *part_dE,
                         int *rounds, int *capped, int max_rounds, int blocks,
                         RoundState *rs, cudaStream_t st)
{
    SweepArgs A;
    A.g = g;
    A.kw = kw;
    A.fc = fc;
    A.chi = chi;
    A.W = W;
    A.U = U;
    A.K = K;
    A.dE = dE;
    A.ntx = (g.nx + TS - 1) / TS;
    A.nty = (g.ny + TS - 1) / TS;
    A.ntz = (g.nz + TS - 1) / TS;
    const int ntiles = A.ntx * A.nty * A.ntz;
    A.act0 = act;
    A.act1 = act + ntiles;
    A.tneg = tneg;
    A.cnt = ctl;
    A.bar = ctl + 3;
    A.err = err;
    A.part_flips = part_flips;
    A.part_dE = part_dE;
    A.rounds_out = rounds;
    A.capped_out = capped;
    A.max_rounds = max_rounds;
    A.use_tma = use_tma;
    // every tile starts active: round 0 is a full pass that finds the band
    cudaMemsetAsync(act, 1, ntiles, st);
    cudaMemsetAsync(act + ntiles, 0, ntiles, st);
    cudaMemsetAsync(ctl, 0, 5 * sizeof(unsigned), st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    CUtensorMap tm;
    if (use_tma) std::memcpy(&tm, tmap, sizeof(tm));
    else std::memset(&tm, 0, sizeof(tm));
    void *args[] = {&tm, &A};
    count_launch();
    cudaError_t e = cudaLaunchCooperativeKernel((void *)k_sweep, dim3(blocks),
                                                dim3(SW_THREADS), args,
                                                sweep_smem_bytes(kw.r), st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_sweep_final<<<1, 1, 0, st>>>(part_flips, part_dE, blocks, rounds, capped, rs);
    return cudaGetLastError();
}

}  // namespace vesis
