// Persistent narrow-band flip sweep (Sec. 3.1, Step 2) for sm_103a.
//
// All flip rounds of one interface relaxation run in a single cooperative
// launch.  The grid is cut into 8^3 tiles; only tiles holding candidate
// cells (a face neighbour with the other label) are active, which is the
// band around the interface the paper restricts the flips to.
//
// Selection rule (the data-parallel form of the min-heap flipping): every
// candidate with dE < 0 gets the 32-bit key bits(float(dE)) (the raw bits of
// a negative float grow as the value falls); other cells get 0.  The grid is
// cut into bricks of edge B (4 when r >= 3, else 2) aligned at index 0; a
// brick's leader is its cell with the largest key, the smallest linear index
// among equal keys, packed as (key << 32) | (2^32 - 1 - index) so that a
// larger word is a better leader.  A leader flips when no other brick's
// leader within Chebyshev distance r is better.  The heap's top always
// flips, flipped cells are more than r apart, the kernel couples none of
// them, and a round lowers the energy by exactly the sum of their dE.
//
// Per round:
//   phase A (one warp per active tile that a flip of the previous round
//     came within r of - the other tiles' keys cannot have changed): the
//     tile's candidate cells are compacted, their flip energies
//     dE = c[s(1-2w) - g0] - s h^3 U are evaluated in FP64 (Eq. dGj1/dGj2),
//     and the tile's brick leaders are written.  A tile without candidates
//     turns inactive.
//   grid barrier
//   phase B (one warp per tile with a negative cell): the packed leaders of
//     the 6^3 bricks around the tile arrive in shared memory together, and
//     each brick leader of the tile is tested against them.  Winners
//     flip; +-q_a q_b q_c is added to W over each winner's window with
//     integer atomics (W stays the exact convolution); the tiles of the
//     winner and of its face neighbours are activated and the tiles within
//     r of it are marked for recomputation.
//   grid barrier; stop when a round flipped nothing.
//
// The grid barrier spins with a bound; on timeout it raises an error flag
// and every block returns.
#include "vesis_internal.cuh"

namespace vesis {

constexpr int TS = 8;             // tile edge
constexpr int TC = TS * TS * TS;  // cells per tile
constexpr int SW_THREADS = 256;
constexpr int NWARP = SW_THREADS / 32;
constexpr long long kSpinLimit = 1ll << 24;   // polls before the barrier gives up
constexpr int kLine = 32;         // words per 128-byte line of the control block
constexpr int kMaxBricksPerTile = 64;         // (8 / 2)^3 for bricks of edge 2
// Bricks per axis a tile's leaders can see: from brick (tile - ceil(r/B)) to
// (tile end + ceil(r/B)); 6 for r <= 8 with B = 4 and for r <= 2 with B = 2.
constexpr int kNbh = 6;
constexpr int kMaxQueue = 512;    // winners per block and round queued for W

// Blocks per SM of the cooperative grid.
#ifndef VESIS_SWEEP_BPS
#define VESIS_SWEEP_BPS 3
#endif

struct SweepArgs {
    GridDesc g;
    KernelW kw;
    FlipConst fc;
    uint8_t *chi;
    uint32_t *W;
    const float *U;
    double *dE;
    unsigned long long *PL;   // packed brick leaders
    uint8_t *act0, *act1, *dirty0, *dirty1, *tneg;
    int ntx, nty, ntz;
    int bs, bsh;        // brick edge and its log2
    int nbx, nby, nbz;  // bricks per axis
    unsigned *cnt;      // [3] flips per round, cycled
    unsigned *bar;      // monotonic arrival counter (own 128-byte line)
    int *err;
    unsigned long long *part_flips;   // [gridDim.x]
    double *part_dE;                  // [gridDim.x]
    int *rounds_out;
    int *capped_out;
    int max_rounds;
};

// Grid barrier on a monotonic arrival counter: barrier number e (1, 2, ...)
// completes when the counter reaches e * gridDim.x.  Arrival is one release
// reduction (it orders the block's earlier writes, which bar.sync has made
// visible to thread 0), the wait a relaxed poll (an acquire load per poll
// would discard the SM's L1 under the blocks still working) closed by one
// acquire fence; no reset is needed.  The poll is bounded and watches the
// error flag every 256 polls; a timeout raises the flag and the caller
// returns.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(const SweepArgs &A, unsigned &target,
                                             int *abort_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(A.bar), "r"(1u)
                     : "memory");
        long long spins = 0;
        while ((int)(ld_relaxed_u32(A.bar) - target) < 0) {
            if ((++spins & 255) == 0 &&
                (spins > kSpinLimit || *(volatile int *)A.err)) {
                atomicExch(A.err, 1);
                *abort_flag = 1;
                break;
            }
            __nanosleep(32);
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
    return *abort_flag == 0;
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
    uint8_t chi[NWARP][(TS + 2) * (TS + 2) * (TS + 2)];   // per-warp label halo
    unsigned long long bmax[NWARP][kMaxBricksPerTile];     // per-warp brick leaders
    uint16_t cl[NWARP][TC];                                // per-warp candidate list
    unsigned long long nbh[NWARP][kNbh * kNbh * kNbh];     // per-warp leader neighbourhood
    long long wl[kMaxQueue];          // this round's winners of the block
    int nwl;
    int abort_flag;                   // set when a grid barrier gave up
    unsigned ncnt;                    // flips of the round, read by thread 0
    int qw[2 * kMaxR + 1];            // 1-D kernel weights
    int list[SW_THREADS];
    int wc[NWARP];
    double e[NWARP];
    unsigned nf[NWARP];
};

// Labels, W, keys, brick leaders and tile flags change under other blocks
// between rounds: every read of them goes to L2 (ld.global.cg), never to a
// stale L1 line.

// Phase A for one tile, one warp.
__device__ __noinline__ void phase_keys_warp(const SweepArgs &A, SweepShared &S, int t,
                                             uint8_t *act_next)
{
    constexpr int E = TS + 2;
    constexpr int EE = E * E * E;
    constexpr int PER = TC / 32;
    constexpr int HB = (EE + 31) / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint8_t *hal = S.chi[wp];
    unsigned long long *bmax = S.bmax[wp];
    const int bpt = TS >> A.bsh;                   // bricks per tile edge
    const int nbt = bpt * bpt * bpt;
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    for (int b = lane; b < nbt; b += 32) bmax[b] = 0ull;
    // labels of the tile and a one-cell halo: all loads of a lane issued
    // before the first store
#pragma unroll
    for (int half = 0; half < 1; ++half) {
        constexpr int HH = HB;
        uint32_t packed[(HH + 3) / 4];
#pragma unroll
        for (int u = 0; u < (HH + 3) / 4; ++u) packed[u] = 0u;
#pragma unroll
        for (int u = 0; u < HH; ++u) {
            const int idx = lane + 32 * (half * HH + u);
            uint32_t v = 0;
            if (idx < EE) {
                const int hz = idx % E, hy = (idx / E) % E, hx = idx / (E * E);
                const int i = i0 - 1 + hx, j = j0 - 1 + hy, k = k0 - 1 + hz;
                if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz)
                    v = __ldcg(A.chi + (long long)i * nyz + (long long)j * g.nz + k);
            }
            packed[u >> 2] |= v << (8 * (u & 3));
        }
#pragma unroll
        for (int u = 0; u < HH; ++u) {
            const int idx = lane + 32 * (half * HH + u);
            if (idx < EE) hal[idx] = (uint8_t)(packed[u >> 2] >> (8 * (u & 3)));
        }
    }
    __syncwarp();
    // candidates, compacted into the warp's list (cell order)
    const unsigned lt = (1u << lane) - 1u;
    int ncand = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int c = lane + 32 * u;
        const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
        bool cand = false;
        if (i0 + x < g.nx && j0 + y < g.ny && k0 + z < g.nz) {
            const int h = ((x + 1) * E + (y + 1)) * E + (z + 1);
            const uint8_t v = hal[h];
            cand = (hal[h - E * E] != v) | (hal[h + E * E] != v) | (hal[h - E] != v) |
                   (hal[h + E] != v) | (hal[h - 1] != v) | (hal[h + 1] != v);
        }
        const unsigned b = __ballot_sync(0xffffffffu, cand);
        if (cand) S.cl[wp][ncand + __popc(b & lt)] = (uint16_t)c;
        ncand += __popc(b);
    }
    __syncwarp();
    // FP64 flip energies of the candidates, 128 at a time: the W and U loads
    // of all four per lane are issued before the first use
    bool neg = false;
    for (int base = 0; base < ncand; base += 128) {
        unsigned Wv[4];
        float Uv[4];
        long long pv[4];
        int cv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = base + 32 * u + lane;
            cv[u] = -1;
            Wv[u] = 0u;
            Uv[u] = 0.f;
            pv[u] = 0;
            if (q < ncand) {
                const int c = S.cl[wp][q];
                const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
                cv[u] = c;
                pv[u] = (long long)(i0 + x) * nyz + (long long)(j0 + y) * g.nz + (k0 + z);
                Wv[u] = __ldcg(A.W + pv[u]);
                Uv[u] = __ldg(A.U + pv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (cv[u] < 0) continue;
            const int c = cv[u];
            const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
            const uint8_t v = hal[((x + 1) * E + (y + 1)) * E + (z + 1)];
            const double e = flip_dE_s(v, Wv[u], Uv[u], A.fc);
            if (e < 0.0) {
                const uint32_t key = __float_as_uint(__double2float_rn(e));
                A.dE[pv[u]] = e;
                neg = true;
                const unsigned long long pk =
                    ((unsigned long long)key << 32) | (0xffffffffull - (unsigned long long)pv[u]);
                const int bb = ((x >> A.bsh) * bpt + (y >> A.bsh)) * bpt + (z >> A.bsh);
                atomicMax(&bmax[bb], pk);
            }
        }
    }
    const bool ca = ncand > 0;
    const bool na = __any_sync(0xffffffffu, neg);
    __syncwarp();
    // brick leaders of this tile (bricks lie inside the tile: B divides 8)
    for (int b = lane; b < nbt; b += 32) {
        const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
        const int gi = (i0 >> A.bsh) + bx, gj = (j0 >> A.bsh) + by, gk = (k0 >> A.bsh) + bz;
        if (gi >= A.nbx || gj >= A.nby || gk >= A.nbz) continue;
        A.PL[((long long)gi * A.nby + gj) * A.nbz + gk] = bmax[b];
    }
    if (lane == 0) {
        act_next[t] = (uint8_t)ca;
        A.tneg[t] = (uint8_t)na;
    }
    __syncwarp();
}

// Phase B for one tile (one warp).  The packed leaders of the bricks its
// leaders' windows can reach are loaded into shared memory with every load
// in flight at once; lane b then tests the leader of the tile's brick b: it
// wins unless another brick's leader within Chebyshev distance r is better
// (a larger packed word).  Returns a bit mask of the winning bricks.
__device__ unsigned long long tile_winners(const SweepArgs &A, unsigned long long *nbh, int t)
{
    constexpr int NN = kNbh * kNbh * kNbh;
    constexpr int PERL = (NN + 31) / 32;
    const int lane = threadIdx.x & 31;
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    const int r = A.kw.r;
    const int bpt = TS >> A.bsh;
    const int reach = (r + A.bs - 1) >> A.bsh;          // ceil(r / B) <= 2
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const int bi0 = (i0 >> A.bsh) - reach, bj0 = (j0 >> A.bsh) - reach, bk0 = (k0 >> A.bsh) - reach;
    unsigned long long v[PERL];
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
        const int q = lane + 32 * u;
        v[u] = 0ull;
        if (q < NN) {
            const int bi = bi0 + q / (kNbh * kNbh), bj = bj0 + (q / kNbh) % kNbh,
                      bk = bk0 + q % kNbh;
            if (bi >= 0 && bj >= 0 && bk >= 0 && bi < A.nbx && bj < A.nby && bk < A.nbz)
                v[u] = __ldcg(A.PL + ((long long)bi * A.nby + bj) * A.nbz + bk);
        }
    }
#pragma unroll
    for (int u = 0; u < PERL; ++u) {
        const int q = lane + 32 * u;
        if (q < NN) nbh[q] = v[u];
    }
    __syncwarp();
    const int nbt = bpt * bpt * bpt;            // 8 (B = 4) or 64 (B = 2)
    unsigned long long mask = 0ull;
    for (int b = lane; b < ((nbt + 31) & ~31); b += 32) {
        bool win = false;
        if (b < nbt) {
            const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
            const unsigned long long pl =
                nbh[((bx + reach) * kNbh + (by + reach)) * kNbh + (bz + reach)];
            if (pl != 0ull) {
                const long long p = (long long)(0xffffffffull - (pl & 0xffffffffull));
                const int ci = (int)(p / nyz), cj = (int)((p / g.nz) % g.ny), ck = (int)(p % g.nz);
                // bricks holding a cell of the window, in neighbourhood coordinates
                const int a0 = (max(ci - r, 0) >> A.bsh) - bi0, a1 = (min(ci + r, g.nx - 1) >> A.bsh) - bi0;
                const int b0 = (max(cj - r, 0) >> A.bsh) - bj0, b1 = (min(cj + r, g.ny - 1) >> A.bsh) - bj0;
                const int c0 = (max(ck - r, 0) >> A.bsh) - bk0, c1 = (min(ck + r, g.nz - 1) >> A.bsh) - bk0;
                win = true;
                for (int a = a0; a <= a1 && win; ++a)
                    for (int bb = b0; bb <= b1 && win; ++bb)
                        for (int c = c0; c <= c1; ++c) {
                            const unsigned long long m = nbh[(a * kNbh + bb) * kNbh + c];
                            if (m <= pl) continue;
                            const long long p2 = (long long)(0xffffffffull - (m & 0xffffffffull));
                            const int i2 = (int)(p2 / nyz), j2 = (int)((p2 / g.nz) % g.ny),
                                      k2 = (int)(p2 % g.nz);
                            if (abs(i2 - ci) <= r && abs(j2 - cj) <= r && abs(k2 - ck) <= r) {
                                win = false;
                                break;
                            }
                        }
            }
        }
        const unsigned m32 = __ballot_sync(0xffffffffu, win);
        mask |= (unsigned long long)m32 << (b - lane);
    }
    __syncwarp();
    return mask;
}

// W window update of one flipped cell, spread over `nthreads` threads with
// index `tid`: +-q_a q_b q_c on every in-grid cell of the cube of half-width
// r around it (integer atomics, so W stays the exact convolution).
__device__ __forceinline__ void add_window(const SweepArgs &A, const int *qw, long long p,
                                           int sgn, int tid, int nthreads)
{
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    const int r = A.kw.r;
    const int w = 2 * r + 1;
    const int i = (int)(p / nyz), j = (int)((p / g.nz) % g.ny), k = (int)(p % g.nz);
    for (int idx = tid; idx < w * w * w; idx += nthreads) {
        const int c = idx % w, b = (idx / w) % w, a = idx / (w * w);
        const int ii = i + a - r, jj = j + b - r, kk = k + c - r;
        if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
        atomicAdd(&A.W[(long long)ii * nyz + (long long)jj * g.nz + kk],
                  (unsigned)(sgn * qw[a] * qw[b] * qw[c]));
    }
}

// Flip of a winner by its warp: label, energy, activation of the tiles of
// the cell and of its face neighbours, recomputation marks for the tiles
// within r.  The W update is queued for the whole block (done after the
// phase); if the queue is full the warp does it at once.
__device__ void flip_winner(const SweepArgs &A, SweepShared &S, long long p,
                            uint8_t *act_next, uint8_t *dirty_next, double &e_warp,
                            unsigned &n_warp)
{
    const int lane = threadIdx.x & 31;
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    const int r = A.kw.r;
    const int i = (int)(p / nyz), j = (int)((p / g.nz) % g.ny), k = (int)(p % g.nz);
    const uint8_t old = __ldcg(A.chi + p);
    int slot = 0;
    if (lane == 0) {
        A.chi[p] = (uint8_t)(1 - old);
        e_warp += __ldcg(A.dE + p);
        n_warp += 1;
        slot = atomicAdd(&S.nwl, 1);
        if (slot < kMaxQueue) S.wl[slot] = old ? -(p + 1) : (p + 1);   // sign: W change
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= kMaxQueue) add_window(A, S.qw, p, old ? -1 : 1, lane, 32);
    if (lane < 7) {
        const int di = (lane == 1) - (lane == 2), dj = (lane == 3) - (lane == 4),
                  dk = (lane == 5) - (lane == 6);
        mark_tile(A, act_next, i + di, j + dj, k + dk);
    }
    // tiles holding a cell within r of the flip: their keys change
    {
        const int ti0 = max(i - r, 0) / TS, ti1 = min(i + r, g.nx - 1) / TS;
        const int tj0 = max(j - r, 0) / TS, tj1 = min(j + r, g.ny - 1) / TS;
        const int tk0 = max(k - r, 0) / TS, tk1 = min(k + r, g.nz - 1) / TS;
        const int mj = tj1 - tj0 + 1, mk = tk1 - tk0 + 1;
        const int mt = (ti1 - ti0 + 1) * mj * mk;
        if (lane < mt) {
            const int ti = ti0 + lane / (mj * mk), tj = tj0 + (lane / mk) % mj, tk = tk0 + lane % mk;
            dirty_next[(ti * A.nty + tj) * A.ntz + tk] = 1;
        }
    }
    __syncwarp();
}

// Collects, in increasing order, this block's tiles t = blockIdx.x + k *
// gridDim.x (k in [base, base + SW_THREADS)) whose flag is set (and, if
// `dirty` is given, whose dirty flag is set too); returns the count (list
// in S.list).  With `nxt` (phase A), own tiles are also prepared for the
// next round: an inactive tile gets nxt = 0 and tneg = 0, an active tile
// that needs no recomputation keeps nxt = 1 and its tneg, and the own
// entries of `clear` (next round's dirty map) are zeroed.
__device__ int gather_tiles(const SweepArgs &A, SweepShared &S, const uint8_t *flags,
                            const uint8_t *dirty, int base, int ntiles, uint8_t *nxt,
                            uint8_t *clear)
{
    const int k = base + threadIdx.x;
    const long long t = (long long)blockIdx.x + (long long)k * gridDim.x;
    bool fl = false;
    if (t < ntiles) {
        const bool act = __ldcg(flags + t) != 0;
        const bool dt = dirty ? (__ldcg(dirty + t) != 0) : true;
        fl = act && dt;
        if (nxt) {
            if (!act) {
                nxt[t] = 0;
                A.tneg[t] = 0;
            } else if (!dt) {
                nxt[t] = 1;
            }
            clear[t] = 0;
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, fl);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    __syncthreads();          // the previous list is no longer read
    if (lane == 0) S.wc[wp] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < NWARP; ++q) {
        if (q < wp) off += S.wc[q];
        tot += S.wc[q];
    }
    if (fl) S.list[off + __popc(b & ((1u << lane) - 1u))] = (int)t;
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(SW_THREADS, VESIS_SWEEP_BPS)
k_sweep(SweepArgs A)
{
    __shared__ SweepShared S;
    const int ntiles = A.ntx * A.nty * A.ntz;
    const int per_block = (ntiles + gridDim.x - 1) / gridDim.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int bpt = TS >> A.bsh;
    for (int a = threadIdx.x; a <= 2 * A.kw.r; a += SW_THREADS) S.qw[a] = A.kw.q[a];
    if (threadIdx.x == 0) {
        S.nwl = 0;
        S.abort_flag = 0;
    }
    __syncthreads();
    unsigned target = 0;      // thread 0: arrivals the next barrier waits for
    unsigned nflip = 0;       // thread 0 only
    double esum = 0.0;        // thread 0 only
    int round = 0, capped = 0;
    for (;;) {
        uint8_t *cur = (round & 1) ? A.act1 : A.act0;
        uint8_t *nxt = (round & 1) ? A.act0 : A.act1;
        uint8_t *dcur = (round & 1) ? A.dirty1 : A.dirty0;
        uint8_t *dnxt = (round & 1) ? A.dirty0 : A.dirty1;
        if (blockIdx.x == 0 && threadIdx.x == 0) A.cnt[(round + 1) % 3] = 0;
        // phase A: one warp per active tile that needs recomputation
        for (int base = 0; base < per_block; base += SW_THREADS) {
            const int n = gather_tiles(A, S, cur, dcur, base, ntiles, nxt, dnxt);
            for (int q = wp; q < n; q += NWARP) phase_keys_warp(A, S, S.list[q], nxt);
        }
        if (!grid_barrier(A, target, &S.abort_flag)) return;
        // phase B: one warp per tile with a negative cell
        double e_warp = 0.0;
        unsigned n_warp = 0;
        for (int base = 0; base < per_block; base += SW_THREADS) {
            const int n = gather_tiles(A, S, A.tneg, nullptr, base, ntiles, nullptr, nullptr);
            for (int q = wp; q < n; q += NWARP) {
                const int t = S.list[q];
                unsigned long long mask = tile_winners(A, S.nbh[wp], t);
                // winners in brick order (the flips of one tile are > r apart)
                while (mask) {
                    const int b = __ffsll((long long)mask) - 1;
                    mask &= mask - 1;
                    int i0, j0, k0;
                    tile_origin(A, t, i0, j0, k0);
                    const int reach = (A.kw.r + A.bs - 1) >> A.bsh;
                    const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
                    const unsigned long long pl =
                        S.nbh[wp][((bx + reach) * kNbh + (by + reach)) * kNbh + (bz + reach)];
                    const long long p = (long long)(0xffffffffull - (pl & 0xffffffffull));
                    flip_winner(A, S, p, nxt, dnxt, e_warp, n_warp);
                }
            }
        }
        if (lane == 0) {
            S.e[wp] = e_warp;
            S.nf[wp] = n_warp;
        }
        __syncthreads();
        // W updates of the queued winners by the whole block
        {
            const int nq = min(S.nwl, kMaxQueue);
            for (int f = 0; f < nq; ++f) {
                const long long v = S.wl[f];
                add_window(A, S.qw, (v > 0 ? v : -v) - 1, v > 0 ? 1 : -1, threadIdx.x,
                           SW_THREADS);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) S.nwl = 0;
        if (threadIdx.x == 0) {
            double te = 0.0;
            unsigned nround = 0;
            for (int q = 0; q < NWARP; ++q) {
                te += S.e[q];
                nround += S.nf[q];
            }
            esum += te;
            nflip += nround;
            if (nround) atomicAdd(&A.cnt[round % 3], nround);
        }
        if (threadIdx.x == 0) S.ncnt = 0;
        if (!grid_barrier(A, target, &S.abort_flag)) return;
        if (threadIdx.x == 0) S.ncnt = ld_acquire_u32(&A.cnt[round % 3]);
        __syncthreads();
        const unsigned n = S.ncnt;
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

int sweep_tiles(const GridDesc &g)
{
    return ((g.nx + TS - 1) / TS) * ((g.ny + TS - 1) / TS) * ((g.nz + TS - 1) / TS);
}

int sweep_brick_edge(int r) { return r >= 3 ? 4 : 2; }

long long sweep_bricks(const GridDesc &g, int r)
{
    const int b = sweep_brick_edge(r);
    return (long long)((g.nx + b - 1) / b) * ((g.ny + b - 1) / b) * ((g.nz + b - 1) / b);
}

cudaError_t sweep_grid_size(int nsm, int *blocks)
{
    int per = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep, SW_THREADS, 0);
    if (e != cudaSuccess) return e;
    per = per > VESIS_SWEEP_BPS ? VESIS_SWEEP_BPS : per;
    *blocks = per * nsm;
    return *blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

int sweep_ctl_words() { return 3 * kLine; }

cudaError_t launch_sweep(const GridDesc &g, const KernelW &kw, const FlipConst &fc,
                         uint8_t *chi, uint32_t *W, const float *U,
                         double *dE, unsigned long long *PL, uint8_t *act,
                         uint8_t *tneg, unsigned *ctl, int *err,
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
    A.dE = dE;
    A.PL = PL;
    A.ntx = (g.nx + TS - 1) / TS;
    A.nty = (g.ny + TS - 1) / TS;
    A.ntz = (g.nz + TS - 1) / TS;
    A.bs = sweep_brick_edge(kw.r);
    A.bsh = A.bs == 4 ? 2 : 1;
    A.nbx = (g.nx + A.bs - 1) / A.bs;
    A.nby = (g.ny + A.bs - 1) / A.bs;
    A.nbz = (g.nz + A.bs - 1) / A.bs;
    const int ntiles = A.ntx * A.nty * A.ntz;
    A.act0 = act;
    A.act1 = act + ntiles;
    A.dirty0 = act + 2 * (long long)ntiles;
    A.dirty1 = act + 3 * (long long)ntiles;
    A.tneg = tneg;
    A.cnt = ctl;
    A.bar = ctl + kLine;
    A.err = err;
    A.part_flips = part_flips;
    A.part_dE = part_dE;
    A.rounds_out = rounds;
    A.capped_out = capped;
    A.max_rounds = max_rounds;
    // every tile starts active and dirty: round 0 is a full pass that finds
    // the band
    cudaMemsetAsync(A.act0, 1, ntiles, st);
    cudaMemsetAsync(A.act1, 0, ntiles, st);
    cudaMemsetAsync(A.dirty0, 1, ntiles, st);
    cudaMemsetAsync(A.dirty1, 0, ntiles, st);
    cudaMemsetAsync(ctl, 0, sweep_ctl_words() * sizeof(unsigned), st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    void *args[] = {&A};
    count_launch();
    cudaError_t e = cudaLaunchCooperativeKernel((void *)k_sweep, dim3(blocks),
                                                dim3(SW_THREADS), args, 0, st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_sweep_final<<<1, 1, 0, st>>>(part_flips, part_dE, blocks, rounds, capped, rs);
    return cudaGetLastError();
}

}  // namespace vesis
