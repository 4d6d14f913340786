// Persistent narrow-band flip sweep (Sec. 3.1, Step 2) for sm_103a.
//
// All flip rounds of one interface relaxation run in a single cooperative
// launch.  The grid is cut into 8^3 tiles; a round only visits tiles that
// hold a cell that may flip or lie near one that just flipped, which keeps
// the work on the band around the interface the paper restricts the flips
// to.
//
// Selection rule (the data-parallel form of the min-heap flipping): every
// candidate cell (a face neighbour has the other label) whose flip lowers
// the energy (dE < 0 in FP64, Eqs. dGj1/dGj2) gets the key float(dE); the
// grid is cut into bricks of edge B (4 when r >= 3, else 2) aligned at
// index 0, and a brick's leader is its cell with the most negative key, the
// smaller linear index among equal keys.  A leader flips when no other
// brick's leader within Chebyshev distance r comes first.  The heap's top
// always flips, flipped cells are more than r apart, the kernel couples
// none of them, and a round lowers the energy by exactly the sum of their
// dE.
//
// A leader is one 64-bit word, larger = first:
//   (magnitude bits of float(dE)) << 33 | (2^32 - 1 - index) << 1 | label,
// zero for a brick without one (PL, one word per brick).
//
// Round k:
//   decide (one warp per tile holding a leader): the words of the 6^3
//     bricks around the tile arrive together; each of the tile's leaders is
//     tested against every other leader within r.  A winner flips its label
//     and adds its dE, and posts itself to every tile within r of it: a
//     16-bit entry (cell within its brick, old label) in the slot of its
//     brick among the 6^3 bricks that tile can see, plus the slot's bit.
//   grid barrier
//   update (one warp per tile that received a winner): W of the tile's own
//     cells gets +-q_a q_b q_c from each posted winner whose window covers
//     them (W stays the exact convolution, and only the warp visiting the
//     tile writes its cells), then the tile's candidates, their dE and its
//     leaders are recomputed.  Tiles no winner reached keep their leaders.
//   grid barrier
// The sweep stops when no tile holds a leader or after max_rounds rounds.
// An opening pass computes every tile's leaders from the starting labels.
//
// Only tiles whose verdict can change are decided: a leader's verdict is a
// function of the leader words within r of it, all inside the 27 tiles
// around its own, so a tile none of whose 27 neighbours (itself included)
// changed a leader word in the last update keeps its last verdict - it
// lost (a winner changes its own tile's words) - and is skipped.  Every
// update that changes one of the tile's words stamps its 27 neighbours with
// the next round; round 0 decides every tile.  The winners, and so the
// rounds and labels, are those of deciding every tile every round.  The
// stamps only pay where warps have several tiles: the updates write them
// while the tiles holding a leader outnumber the grid's warps (a count all
// blocks read alike), and a block reads them only after such an update and
// when its own leader tiles outnumber its warps (deciding an unstamped tile
// is harmless).
//
// The grid barrier spins with a bound; on timeout it raises an error flag
// and every block returns.
#include <vector>

#include "vesis_internal.cuh"

namespace vesis {

constexpr int TS = 8;             // tile edge
#ifndef VESIS_SWEEP_THREADS
#define VESIS_SWEEP_THREADS 512
#endif
constexpr int SW_THREADS = VESIS_SWEEP_THREADS;
constexpr int NWARP = SW_THREADS / 32;
constexpr int kLine = 32;         // words per 128-byte line of the control block
constexpr int kMaxBricksPerTile = 64;         // (8 / 2)^3 for bricks of edge 2
constexpr int kHaloRows = (TS + 2) * (TS + 2);
// Bricks per axis a tile can see: the tile's own (8 / B) and ceil(r / B) on
// each side; 6 for r <= 8 with B = 4 and for r <= 2 with B = 2.  Leaders
// within r of a tile, and the rivals of a tile's own leaders, all lie there.
constexpr int kNbh = 6;
constexpr int kNbh3 = kNbh * kNbh * kNbh;
// Winners within r of a tile are more than r apart inside a box of edge
// 8 + 2r: at most ceil((8 + 2r) / (r + 1))^3 <= 125 of them.
constexpr int kMaxWin = 128;
// Tiles a thread examines per pass when a block lists its tiles: one pass
// lists up to SW_THREADS * kGatherPer of them.
constexpr int kGatherPer = 4;
constexpr int kListCap = SW_THREADS * kGatherPer;
// Posting area of a tile: 216 16-bit slots and an 8-word slot bitmap.
constexpr int kPostBytes = 512;
constexpr int kPostMaskOff = 448;

// Blocks per SM of the cooperative grid (upper bound; shared memory and
// registers may allow fewer).
#ifndef VESIS_SWEEP_BPS
#define VESIS_SWEEP_BPS 1
#endif
// A block keeps one bit per own tile (holds a leader) in shared memory:
// up to 32768 own tiles, more than a grid of 2^31 cells gives any block.
constexpr int kOwnWords = 1024;

struct SweepArgs {
    GridDesc g;
    KernelW kw;
    double cD;          // c_N: dE = c_N N - s h^3 U
    double h3;
    int qc3;            // k0, the kernel's centre weight
    int ksum;           // S, the sum of all kernel weights
    const int *k3;      // full stencil (device) or NULL for the product kernel
    uint8_t *chi;
    uint32_t *W;
    const float *U;
    double *dE;
    unsigned long long *PL;   // leader word per brick
    uint8_t *PO;              // leader cell within its brick: di | dj << 2 | dk << 4
    unsigned *CB;             // labels, one bit per cell: word w of column (i, j)
                              // at (w nx + i) ny + j (a tile's halo words adjoin)
    int nzw;
    uint8_t *post;            // posting area per tile (kPostBytes)
    uint8_t *upd;             // tile received a winner this round
    int *dirty;               // per tile: the round whose decide must visit it
    int ntx, nty, ntz;
    int bs, bsh;        // brick edge and its log2
    int reach;          // ceil(r / B)
    int nbx, nby, nbz;  // bricks per axis
    int vec;            // rows of 8 W and U values may be loaded as vectors
    unsigned *nlead;    // tiles holding a leader (kept current by the updates)
    unsigned *bar;      // monotonic arrival counter (own 128-byte line)
    int *err;
    unsigned long long *part_flips;   // [gridDim.x]
    double *part_dE;                  // [gridDim.x]
    unsigned long long *part_tiles;   // [2][gridDim.x]: tiles decided, tiles updated
    int *rounds_out;
    int *capped_out;
    int max_rounds;
    long long spin_limit;     // polls before a barrier wait gives up
    int stamps;               // decide stamps: -1 by the leader count, 0 never, 1 always
    RoundState *rs;           // this system's totals (multi-system sweep)
    double *tile_dE;          // per tile: its winners' dE, summed over rounds (multi)
    unsigned *tile_nf;        // per tile: its flips (multi)
};

// Per-warp shared memory; the decide and update phases use it in turn.
struct WarpMem {
    union {
        struct {
            unsigned long long w[kNbh3];   // leader words of the 6^3 bricks
            unsigned c[kNbh3];             // their cells, 5 bits per axis
            unsigned long long cw[kNbh3];  // the non-zero words, compacted
            unsigned cc[kNbh3];            // and their cells
        } d;
        struct {
            unsigned cW[512];              // candidates: W
            float cU[512];                 //             U
            unsigned short cP[512];        //             tile cell | label << 9
            unsigned hr[kHaloRows];        // label bits of the halo rows (bit 0: z = -1)
            unsigned win[kMaxWin];         // winners: tile coords + 8 (5 bits each) | label << 15
            unsigned long long bmax[kMaxBricksPerTile];   // new leader per brick
        } u;
    };
};

// Grid barrier on a monotonic arrival counter: barrier number e (1, 2, ...)
// completes when the counter reaches e * gridDim.x.  Arrival is one release
// reduction (it orders the block's earlier writes, which bar.sync has made
// visible to thread 0), the wait a relaxed poll (an acquire load per poll
// would discard the SM's L1 under the blocks still working) closed by one
// acquire load of the counter, which reads the completed count and so
// synchronises with every arrival's release (a barrier alone measured 1.16
// us against 1.26 with a closing acquire fence); no reset is needed.  The poll is bounded (A.spin_limit
// polls; 0 gives up at the first poll that finds the barrier open) and
// watches the error flag every 256 polls; a timeout raises the flag and the
// caller returns.
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, long long spin_limit,
                                             unsigned &target, int *abort_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(bar), "r"(1u)
                     : "memory");
        long long spins = 0;
        while ((int)(ld_relaxed_u32(bar) - target) < 0) {
            if (++spins > spin_limit ||
                ((spins & 255) == 0 && *(volatile int *)err)) {
                atomicExch(err, 1);
                *abort_flag = 1;
                break;
            }
            __nanosleep(32);
        }
        (void)ld_acquire_u32(bar);
    }
    __syncthreads();
    return *abort_flag == 0;
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

// Cell (ci, cj, ck) of the leader word w of brick (bx, by, bz), found from
// its linear index without a division: the offset from the brick's first
// cell is di * nyz + dj * nz + dk with 0 <= di, dj, dk < B.
__device__ __forceinline__ void leader_cell(const SweepArgs &A, unsigned long long w,
                                            int bx, int by, int bz, int &ci, int &cj,
                                            int &ck)
{
    const long long nyz = (long long)A.g.ny * A.g.nz;
    const long long p = (long long)(0xffffffffull - ((w >> 1) & 0xffffffffull));
    ci = bx << A.bsh;
    cj = by << A.bsh;
    ck = bz << A.bsh;
    long long d = p - ((long long)ci * nyz + (long long)cj * A.g.nz + ck);
    for (int s = 1; s < A.bs; ++s)
        if (d >= nyz) {
            d -= nyz;
            ++ci;
        }
    for (int s = 1; s < A.bs; ++s)
        if (d >= A.g.nz) {
            d -= A.g.nz;
            ++cj;
        }
    ck += (int)d;
}

__device__ __forceinline__ void red_or(unsigned *p, unsigned v)
{
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_add(unsigned *p, unsigned v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// 16-byte asynchronous global -> shared copy through L2 (zero fill when
// !valid), and the wait for this thread's copies.
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(dst), "l"(src), "r"(valid ? 16 : 0) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Labels, W, dE, leader words, postings and tile flags change under other
// warps and blocks between phases: every read of them goes to L2
// (ld.global.cg), never to a stale L1 line.

// Decide phase for tile t (one warp).
__device__ __forceinline__ void tile_decide(const SweepArgs &A, WarpMem &M, int t,
                                            double &e_lane, unsigned &n_lane)
{
    const int lane = threadIdx.x & 31;
    const GridDesc &g = A.g;
    const int r = A.kw.r, bsh = A.bsh, reach = A.reach;
    const int bpt = TS >> bsh;
    const int nbt = bpt * bpt * bpt;
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const int nbx0 = (i0 >> bsh) - reach, nby0 = (j0 >> bsh) - reach, nbz0 = (k0 >> bsh) - reach;
    constexpr int PER = (kNbh3 + 31) / 32;
    unsigned long long v[PER];
    unsigned off[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int q = lane + 32 * u;
        v[u] = 0ull;
        off[u] = 0u;
        if (q < kNbh3) {
            const int bx = nbx0 + q / (kNbh * kNbh), by = nby0 + (q / kNbh) % kNbh,
                      bz = nbz0 + q % kNbh;
            if (bx >= 0 && by >= 0 && bz >= 0 && bx < A.nbx && by < A.nby && bz < A.nbz) {
                const long long o = ((long long)bx * A.nby + by) * A.nbz + bz;
                v[u] = __ldcg(A.PL + o);
                off[u] = __ldcg(A.PO + o);
            }
        }
    }
    // leader cells relative to the neighbourhood's first cell; the non-zero
    // words compacted for the scans below
    int m = 0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int q = lane + 32 * u;
        unsigned c = 0u;
        if (v[u] != 0ull) {
            const int bx = q / (kNbh * kNbh), by = (q / kNbh) % kNbh, bz = q % kNbh;
            c = (unsigned)(bx * A.bs + (int)(off[u] & 3u)) |
                ((unsigned)(by * A.bs + (int)((off[u] >> 2) & 3u)) << 5) |
                ((unsigned)(bz * A.bs + (int)((off[u] >> 4) & 3u)) << 10);
        }
        if (q < kNbh3) {
            M.d.w[q] = v[u];
            M.d.c[q] = c;
        }
        const unsigned bm = __ballot_sync(0xffffffffu, v[u] != 0ull);
        if (v[u] != 0ull) {
            const int pos = m + __popc(bm & ((1u << lane) - 1u));
            M.d.cw[pos] = v[u];
            M.d.cc[pos] = c;
        }
        m += __popc(bm);
    }
    __syncwarp();
    // verdicts: a leader of the tile wins unless another within r is better.
    // G lanes share one of the tile's bricks and split the scan of the
    // compacted words between them.
    unsigned long long wmask = 0ull;
    {
        const int G = nbt >= 32 ? 1 : 32 / nbt;      // 4 for 8 bricks
        const int P = 32 / G;                         // bricks per pass
        const int gl = lane / G, sub = lane - gl * G;
        for (int b0 = 0; b0 < nbt; b0 += P) {
            const int b = b0 + gl;
            unsigned long long L = 0ull;
            int lx = 0, ly = 0, lz = 0;
            if (b < nbt) {
                const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
                const int o = ((reach + bx) * kNbh + (reach + by)) * kNbh + (reach + bz);
                L = M.d.w[o];
                const unsigned lc = M.d.c[o];
                lx = lc & 31;
                ly = (lc >> 5) & 31;
                lz = (lc >> 10) & 31;
            }
            bool lose = false;
            if (L != 0ull) {
                // branch-free and unrolled, so that several shared-memory
                // loads are in flight at once
#pragma unroll 4
                for (int q = sub; q < m; q += G) {
                    const unsigned long long w = M.d.cw[q];
                    const unsigned c = M.d.cc[q];
                    const int ox = c & 31, oy = (c >> 5) & 31, oz = (c >> 10) & 31;
                    lose |= (w > L) & (abs(ox - lx) <= r) & (abs(oy - ly) <= r) &
                            (abs(oz - lz) <= r);
                }
            }
            const unsigned lb = __ballot_sync(0xffffffffu, lose);
            const unsigned gm = (G == 32) ? 0xffffffffu : ((1u << G) - 1u);
            const bool win = L != 0ull && sub == 0 && ((lb >> (gl * G)) & gm) == 0u;
            const unsigned wb = __ballot_sync(0xffffffffu, win);
            for (int q = 0; q < P && b0 + q < nbt; ++q)
                if ((wb >> (q * G)) & 1u) wmask |= 1ull << (b0 + q);
        }
    }
    if (wmask == 0ull) return;
    // winners: flip and fetch dE (added at the end), post to every tile
    // within r
    double dv[2] = {0.0, 0.0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int b = lane + 32 * h;
        if (b >= nbt || !((wmask >> b) & 1ull)) continue;
        const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
        const int o = ((reach + bx) * kNbh + (reach + by)) * kNbh + (reach + bz);
        const unsigned long long L = M.d.w[o];
        const unsigned lc = M.d.c[o];
        const int ci = nbx0 * A.bs + (int)(lc & 31), cj = nby0 * A.bs + (int)((lc >> 5) & 31),
                  ck = nbz0 * A.bs + (int)((lc >> 10) & 31);
        const long long p = (long long)(0xffffffffull - ((L >> 1) & 0xffffffffull));
        A.chi[p] = (uint8_t)(1u - (unsigned)(L & 1ull));
        asm volatile("red.relaxed.gpu.global.xor.b32 [%0], %1;"
                     :: "l"(A.CB + ((long long)(ck >> 5) * g.nx + ci) * g.ny + cj),
                        "r"(1u << (ck & 31)) : "memory");
        dv[h] = __ldcg(A.dE + p);
        n_lane += 1u;
    }
    unsigned long long rest = wmask;
    while (rest) {
        const int b = __ffsll((long long)rest) - 1;
        rest &= rest - 1;
        const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
        const int o = ((reach + bx) * kNbh + (reach + by)) * kNbh + (reach + bz);
        const unsigned long long L = M.d.w[o];
        const unsigned lc = M.d.c[o];
        const int ci = (nbx0 * A.bs) + (int)(lc & 31), cj = (nby0 * A.bs) + (int)((lc >> 5) & 31),
                  ck = (nbz0 * A.bs) + (int)((lc >> 10) & 31);
        const unsigned entry = (unsigned)(ci & (A.bs - 1)) | ((unsigned)(cj & (A.bs - 1)) << 2) |
                               ((unsigned)(ck & (A.bs - 1)) << 4) | ((unsigned)(L & 1ull) << 6);
        const int ti0 = max(ci - r, 0) / TS, ti1 = min(ci + r, g.nx - 1) / TS;
        const int tj0 = max(cj - r, 0) / TS, tj1 = min(cj + r, g.ny - 1) / TS;
        const int tk0 = max(ck - r, 0) / TS, tk1 = min(ck + r, g.nz - 1) / TS;
        if (lane < 27) {
            const int ta = ti0 + lane / 9, tb = tj0 + (lane / 3) % 3, tc = tk0 + lane % 3;
            if (ta <= ti1 && tb <= tj1 && tc <= tk1) {
                const int tt = (ta * A.nty + tb) * A.ntz + tc;
                // the winner's brick among the 6^3 bricks tile tt sees
                const int sx = (ci >> bsh) - ((ta * TS) >> bsh) + reach;
                const int sy = (cj >> bsh) - ((tb * TS) >> bsh) + reach;
                const int sz = (ck >> bsh) - ((tc * TS) >> bsh) + reach;
                const int slot = (sx * kNbh + sy) * kNbh + sz;
                uint8_t *pa = A.post + (size_t)tt * kPostBytes;
                reinterpret_cast<unsigned short *>(pa)[slot] = (unsigned short)entry;
                red_or(reinterpret_cast<unsigned *>(pa + kPostMaskOff) + (slot >> 5),
                       1u << (slot & 31));
                A.upd[tt] = 1;
            }
        }
    }
    e_lane += dv[0];
    e_lane += dv[1];
}

// Update phase for tile t (one warp).  first: the opening pass (no
// winners; every tile computes its leaders).  mark >= 0: if a leader word
// of the tile changes, the 27 tiles around it (itself included) are
// stamped with mark, the round whose decide must visit them.
template <bool STENCIL>
__device__ __forceinline__ bool tile_update(const SweepArgs &A, WarpMem &M, const int *qw,
                                            const int *kt,
                                            int t, bool first, int mark)
{
    const int lane = threadIdx.x & 31;
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    const int r = A.kw.r, bsh = A.bsh, reach = A.reach;
    const int bpt = TS >> bsh;
    const int nbt = bpt * bpt * bpt;
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const int zlim = min(TS, g.nz - k0);
    const unsigned zmask = (1u << zlim) - 1u;

    // ---------------------------------------------------------- loads
    // All of a lane's loads are issued before the first use.  W and U of the
    // tile's own cells: rows rho = lane + 32 m, (x, y) = (rho >> 3, rho & 7).
    // With 8-cell rows in 16-byte pieces (vec) they pass through the warp's
    // candidate area in shared memory, consecutive lanes on consecutive
    // pieces (two lanes per 32-byte row), so that each copy instruction
    // reads whole sectors; otherwise each lane loads its rows itself.
    unsigned Wr[2][TS];
    float Ur[2][TS];
    bool rowok[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int rho = lane + 32 * m;
        rowok[m] = (i0 + (rho >> 3) < g.nx) && (j0 + (rho & 7) < g.ny);
#pragma unroll
        for (int z = 0; z < TS; ++z) {
            Wr[m][z] = 0u;
            Ur[m][z] = 0.f;
        }
    }
    const unsigned sW = (unsigned)__cvta_generic_to_shared(M.u.cW);
    const unsigned sU = (unsigned)__cvta_generic_to_shared(M.u.cU);
    if (A.vec) {
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            const int c = lane + 32 * c4;            // piece c: row c >> 1, half c & 1
            const int rho = c >> 1;
            const bool ok = (i0 + (rho >> 3) < g.nx) && (j0 + (rho & 7) < g.ny);
            const long long o = ok ? (long long)(i0 + (rho >> 3)) * nyz +
                                         (long long)(j0 + (rho & 7)) * g.nz + k0 + 4 * (c & 1)
                                   : 0;
            cp_async16(sW + 16u * (unsigned)c, A.W + o, ok);
            cp_async16(sU + 16u * (unsigned)c, A.U + o, ok);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rho = lane + 32 * m;
            if (!rowok[m]) continue;
            const long long o = (long long)(i0 + (rho >> 3)) * nyz +
                                (long long)(j0 + (rho & 7)) * g.nz + k0;
#pragma unroll
            for (int z = 0; z < TS; ++z)
                if (z < zlim) {
                    Wr[m][z] = __ldcg(A.W + o + z);
                    Ur[m][z] = __ldg(A.U + o + z);
                }
        }
    }
    // halo label rows from the bit copy: row h = hx * 10 + hy is the cell
    // column (i0 - 1 + hx, j0 - 1 + hy); bit z + 1 is cell k0 + z, z = -1..8.
    // Cells k0..k0 + 7 share word k0 / 32 (k0 is a multiple of 8); cell k0 - 1
    // or k0 + 8 sits in the word before or after when k0 % 32 is 0 or 24.
    // Bits past the end of a row are zero (solvent, as outside the box).
    unsigned hb[4];
    {
        const int sh = k0 & 31, wm = k0 >> 5;
        const bool need_lo = sh == 0 && k0 > 0, need_hi = sh == 24 && k0 + TS < g.nz;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int h = lane + 32 * u;
            hb[u] = 0u;
            if (h < kHaloRows) {
                const int i = i0 - 1 + h / 10, j = j0 - 1 + h % 10;
                if (i >= 0 && j >= 0 && i < g.nx && j < g.ny) {
                    const unsigned *col = A.CB + (long long)i * g.ny + j;
                    const long long pl = (long long)g.nx * g.ny;     // words per plane
                    const unsigned vm = __ldcg(col + wm * pl);
                    const unsigned vl = need_lo ? __ldcg(col + (wm - 1) * pl) : 0u;
                    const unsigned vh = need_hi ? __ldcg(col + (wm + 1) * pl) : 0u;
                    const unsigned lo = sh == 0 ? (vl >> 31) : ((vm >> (sh - 1)) & 1u);
                    const unsigned hi = sh == 24 ? (vh & 1u) : ((vm >> (sh + 8)) & 1u);
                    hb[u] = lo | (((vm >> sh) & 0xffu) << 1) | (hi << 9);
                }
            }
        }
    }
    // the tile's leader words before this update (brick b = lane + 32 h)
    unsigned long long oldw[2] = {0ull, 0ull};
    if (mark >= 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b = lane + 32 * h;
            if (b >= nbt) continue;
            const int gx = (i0 >> bsh) + b / (bpt * bpt), gy = (j0 >> bsh) + (b / bpt) % bpt,
                      gz = (k0 >> bsh) + b % bpt;
            if (gx < A.nbx && gy < A.nby && gz < A.nbz)
                oldw[h] = __ldcg(A.PL + ((long long)gx * A.nby + gy) * A.nbz + gz);
        }
    }
    // posted winners: slot bitmap (lanes 0..7) and the 216 slots (lanes x 4 per u64)
    uint8_t *pa = A.post + (size_t)t * kPostBytes;
    unsigned pmask = 0u;
    unsigned long long pslot[2] = {0ull, 0ull};
    if (!first) {
        if (lane < 8) pmask = __ldcg(reinterpret_cast<const unsigned *>(pa + kPostMaskOff) + lane);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int q = lane + 32 * m;            // u64 q holds slots 4q .. 4q + 3
            if (q < kNbh3 / 4) pslot[m] = __ldcg(reinterpret_cast<const unsigned long long *>(pa) + q);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int h = lane + 32 * u;
        if (h < kHaloRows) M.u.hr[h] = hb[u];
    }
    if (A.vec) {      // the staged rows into registers before the area is reused
        cp_async_wait_all();
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rho = lane + 32 * m;
            const uint4 w0 = reinterpret_cast<const uint4 *>(M.u.cW)[2 * rho];
            const uint4 w1 = reinterpret_cast<const uint4 *>(M.u.cW)[2 * rho + 1];
            const float4 u0 = reinterpret_cast<const float4 *>(M.u.cU)[2 * rho];
            const float4 u1 = reinterpret_cast<const float4 *>(M.u.cU)[2 * rho + 1];
            Wr[m][0] = w0.x; Wr[m][1] = w0.y; Wr[m][2] = w0.z; Wr[m][3] = w0.w;
            Wr[m][4] = w1.x; Wr[m][5] = w1.y; Wr[m][6] = w1.z; Wr[m][7] = w1.w;
            Ur[m][0] = u0.x; Ur[m][1] = u0.y; Ur[m][2] = u0.z; Ur[m][3] = u0.w;
            Ur[m][4] = u1.x; Ur[m][5] = u1.y; Ur[m][6] = u1.z; Ur[m][7] = u1.w;
        }
        __syncwarp();
    }

    // ------------------------------------------------- posted winners
    int nw = 0;
    if (!first) {
        // the bitmap is consumed: clear it for the next round's postings
        if (lane < 8 && pmask) reinterpret_cast<unsigned *>(pa + kPostMaskOff)[lane] = 0u;
        // slot values to shared memory (reuse the candidate W list as scratch)
        unsigned short *ps = reinterpret_cast<unsigned short *>(M.u.cW);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int q = lane + 32 * m;
            if (q < kNbh3 / 4) reinterpret_cast<unsigned long long *>(ps)[q] = pslot[m];
        }
        __syncwarp();
        // decode the set slots of each bitmap word (lane l < 7 owns word l)
        const int cnt = __popc(pmask);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        nw = __shfl_sync(0xffffffffu, incl, 7);
        int pos = incl - cnt;
        unsigned mm = pmask;
        while (mm) {
            const int bit = __ffs(mm) - 1;
            mm &= mm - 1;
            const int slot = lane * 32 + bit;
            const unsigned e = ps[slot];
            const int sx = slot / (kNbh * kNbh), sy = (slot / kNbh) % kNbh, sz = slot % kNbh;
            // winner cell relative to the tile origin
            const int wx = (sx - reach) * A.bs + (int)(e & 3u);
            const int wy = (sy - reach) * A.bs + (int)((e >> 2) & 3u);
            const int wz = (sz - reach) * A.bs + (int)((e >> 4) & 3u);
            if (pos < kMaxWin)
                M.u.win[pos] = (unsigned)(wx + 8) | ((unsigned)(wy + 8) << 5) |
                               ((unsigned)(wz + 8) << 10) | (((e >> 6) & 1u) << 15);
            ++pos;
        }
        nw = min(nw, kMaxWin);
        __syncwarp();
        // W of the tile's own cells
        bool changed[2] = {false, false};
        for (int e = 0; e < nw; ++e) {
            const unsigned wv = M.u.win[e];
            const int wx = (int)(wv & 31) - 8, wy = (int)((wv >> 5) & 31) - 8,
                      wz = (int)((wv >> 10) & 31) - 8;
            const int sgn = ((wv >> 15) & 1u) ? -1 : 1;   // solute -> solvent lowers W
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int rho = lane + 32 * m;
                const int ax = (rho >> 3) - wx, ay = (rho & 7) - wy;
                if (abs(ax) > r || abs(ay) > r) continue;
                changed[m] = true;
                if (STENCIL) {      // full stencil: the row of weights at (ax, ay)
                    const int *wr = kt + ((ax + r) * (2 * r + 1) + (ay + r)) * (2 * r + 1) + r;
#pragma unroll
                    for (int z = 0; z < TS; ++z) {
                        const int az = z - wz;
                        if (abs(az) <= r) Wr[m][z] += (unsigned)(sgn * wr[az]);
                    }
                } else {
                    const int qxy = sgn * qw[ax + r] * qw[ay + r];
#pragma unroll
                    for (int z = 0; z < TS; ++z) {
                        const int az = z - wz;
                        if (abs(az) <= r) Wr[m][z] += (unsigned)(qxy * qw[az + r]);
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            if (!changed[m] || !rowok[m]) continue;
            const int rho = lane + 32 * m;
            const long long o = (long long)(i0 + (rho >> 3)) * nyz +
                                (long long)(j0 + (rho & 7)) * g.nz + k0;
            if (A.vec) {
                uint4 *wp = reinterpret_cast<uint4 *>(A.W + o);
                wp[0] = make_uint4(Wr[m][0], Wr[m][1], Wr[m][2], Wr[m][3]);
                wp[1] = make_uint4(Wr[m][4], Wr[m][5], Wr[m][6], Wr[m][7]);
            } else {
#pragma unroll
                for (int z = 0; z < TS; ++z)
                    if (z < zlim) A.W[o + z] = Wr[m][z];
            }
        }
        __syncwarp();
    }

    // ------------------------------------ candidates, dE, new leaders
    for (int b = lane; b < nbt; b += 32) M.u.bmax[b] = 0ull;
    int ncand = 0;
    {
        unsigned cm[2], lab[2];
        int cnt = 0;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rho = lane + 32 * m;
            const int x = rho >> 3, y = rho & 7;
            const unsigned c = M.u.hr[(x + 1) * 10 + (y + 1)];
            const unsigned d = (c ^ M.u.hr[x * 10 + (y + 1)]) |
                               (c ^ M.u.hr[(x + 2) * 10 + (y + 1)]) |
                               (c ^ M.u.hr[(x + 1) * 10 + y]) |
                               (c ^ M.u.hr[(x + 1) * 10 + (y + 2)]) |
                               (c ^ (c << 1)) | (c ^ (c >> 1));
            cm[m] = rowok[m] ? (d >> 1) & zmask : 0u;
            lab[m] = (c >> 1) & 0xffu;
            cnt += __popc(cm[m]);
        }
        int incl = cnt;   // inclusive warp scan of the counts
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        ncand = __shfl_sync(0xffffffffu, incl, 31);
        int pos = incl - cnt;
        __syncwarp();     // the slot scratch in cW is no longer read
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rho = lane + 32 * m;
#pragma unroll
            for (int z = 0; z < TS; ++z) {
                if ((cm[m] >> z) & 1u) {
                    M.u.cW[pos] = Wr[m][z];
                    M.u.cU[pos] = Ur[m][z];
                    M.u.cP[pos] = (unsigned short)((rho << 3) | z | (((lab[m] >> z) & 1u) << 9));
                    ++pos;
                }
            }
        }
    }
    __syncwarp();
    // dE = c [s (1 - 2w) - g0] - s h^3 U with s = 1 - 2 chi, w = W / S and
    // g0 = k0 / S (S the sum of the kernel's weights, k0 its centre weight):
    // the bracket is the integer N = s (S - 2W) - k0 over S, so
    // c * bracket = c_N N with c_N = c / S and one rounding.
    for (int q0 = 0; q0 < ncand; q0 += 32) {
        const int q = q0 + lane;
        if (q >= ncand) continue;
        const unsigned Wv = M.u.cW[q];
        const float Uv = M.u.cU[q];
        const unsigned cp = M.u.cP[q];
        const int x = (cp >> 6) & 7, y = (cp >> 3) & 7, z = cp & 7;
        const bool solute = (cp >> 9) & 1u;
        const int base = A.ksum - 2 * (int)Wv;
        const int N = (solute ? -base : base) - A.qc3;
        const double t1 = __dmul_rn(A.cD, (double)N);
        const double t2 = __dmul_rn(A.h3, (double)Uv);
        const double e = __dadd_rn(t1, solute ? t2 : -t2);
        if (e < 0.0) {
            const long long p =
                (long long)(i0 + x) * nyz + (long long)(j0 + y) * g.nz + (k0 + z);
            A.dE[p] = e;
            const unsigned key = __float_as_uint(__double2float_rn(e)) & 0x7fffffffu;
            const unsigned long long w = ((unsigned long long)key << 33) |
                                         ((0xffffffffull - (unsigned long long)p) << 1) |
                                         (unsigned long long)solute;
            atomicMax(&M.u.bmax[((x >> bsh) * bpt + (y >> bsh)) * bpt + (z >> bsh)], w);
        }
    }
    __syncwarp();
    bool any = false, changed = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int b = lane + 32 * h;
        if (b >= nbt) continue;
        const int bx = b / (bpt * bpt), by = (b / bpt) % bpt, bz = b % bpt;
        const int gx = (i0 >> bsh) + bx, gy = (j0 >> bsh) + by, gz = (k0 >> bsh) + bz;
        if (gx >= A.nbx || gy >= A.nby || gz >= A.nbz) continue;
        const unsigned long long w = M.u.bmax[b];
        const long long o = ((long long)gx * A.nby + gy) * A.nbz + gz;
        changed |= w != oldw[h];
        A.PL[o] = w;
        if (w != 0ull) {
            int ci, cj, ck;
            leader_cell(A, w, gx, gy, gz, ci, cj, ck);
            A.PO[o] = (uint8_t)((ci & (A.bs - 1)) | ((cj & (A.bs - 1)) << 2) |
                                ((ck & (A.bs - 1)) << 4));
        }
        any |= w != 0ull;
    }
    if (mark >= 0 && __any_sync(0xffffffffu, changed) && lane < 27) {
        const int tk = t % A.ntz, tj = (t / A.ntz) % A.nty, ti = t / (A.ntz * A.nty);
        const int a = ti + lane / 9 - 1, b = tj + (lane / 3) % 3 - 1, c = tk + lane % 3 - 1;
        if (a >= 0 && b >= 0 && c >= 0 && a < A.ntx && b < A.nty && c < A.ntz)
            A.dirty[(a * A.nty + b) * A.ntz + c] = mark;
    }
    return __any_sync(0xffffffffu, any);
}

struct SweepShared {
    unsigned own[kOwnWords];   // own tile j = (t - blockIdx.x) / gridDim.x holds a leader
    int list[kListCap];
    int wc[NWARP];
    int qw[2 * kMaxR + 1];
    double e[NWARP];
    unsigned nf[NWARP];
    unsigned ncnt;
    int nown;                  // own tiles holding a leader
    int abort_flag;
};

// Lists this block's tiles t = blockIdx.x + j * gridDim.x, j in [base,
// base + kListCap), for which pick(j, t) holds, in a fixed order (thread i
// examines j = base + i + c * SW_THREADS, c < kGatherPer, and its picks
// follow those of threads i' < i); returns the count (list in S.list).
// pick is called once per j < limit with t < ntiles; it may clear a flag.
template <class Pick>
__device__ int list_tiles(SweepShared &S, int base, int limit, long long ntiles, Pick pick)
{
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (limit - base <= SW_THREADS) {    // one tile per thread: a ballot orders them
        const int j = base + threadIdx.x;
        const long long t = (long long)blockIdx.x + (long long)j * gridDim.x;
        const bool fl = j < limit && t < ntiles && pick(j, (int)t);
        const unsigned b = __ballot_sync(0xffffffffu, fl);
        __syncthreads();      // the previous list is no longer read
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
    unsigned m = 0u;
#pragma unroll
    for (int c = 0; c < kGatherPer; ++c) {
        const int j = base + threadIdx.x + c * SW_THREADS;
        const long long t = (long long)blockIdx.x + (long long)j * gridDim.x;
        if (j < limit && t < ntiles && pick(j, (int)t)) m |= 1u << c;
    }
    const int cnt = __popc(m);
    int incl = cnt;   // inclusive warp scan of the counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    __syncthreads();          // the previous list is no longer read
    if (lane == 31) S.wc[wp] = incl;
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < NWARP; ++q) {
        if (q < wp) off += S.wc[q];
        tot += S.wc[q];
    }
    int pos = off + incl - cnt;
#pragma unroll
    for (int c = 0; c < kGatherPer; ++c)
        if ((m >> c) & 1u)
            S.list[pos++] = (int)(blockIdx.x + (long long)(base + threadIdx.x + c * SW_THREADS) *
                                                   gridDim.x);
    __syncthreads();
    return tot;
}

// Whether own tile j holds a leader.
__device__ __forceinline__ bool own_bit(const SweepShared &S, int j)
{
    return (S.own[j >> 5] >> (j & 31)) & 1u;
}

// Records whether own tile t holds a leader, keeping the global count.
__device__ __forceinline__ void set_own(const SweepArgs &A, SweepShared &S, int t, bool now)
{
    const int j = (int)((t - (int)blockIdx.x) / (int)gridDim.x);
    const unsigned bit = 1u << (j & 31);
    const bool old = (S.own[j >> 5] & bit) != 0u;
    if (now == old) return;
    if (now) atomicOr(&S.own[j >> 5], bit);
    else atomicAnd(&S.own[j >> 5], ~bit);
    atomicAdd(&S.nown, now ? 1 : -1);
    red_add(A.nlead, now ? 1u : 0xffffffffu);
}

template <bool STENCIL>
__global__ void __launch_bounds__(SW_THREADS, 1)
k_sweep(SweepArgs A)
{
    __shared__ SweepShared S;
    extern __shared__ __align__(16) unsigned char dyn[];
    WarpMem *WM = reinterpret_cast<WarpMem *>(dyn);
    const int ntiles = A.ntx * A.nty * A.ntz;
    const int per_block = (ntiles + gridDim.x - 1) / gridDim.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    WarpMem &M = WM[wp];
    // the full stencil, if any, follows the warps' areas
    int *kt = STENCIL ? reinterpret_cast<int *>(dyn + NWARP * sizeof(WarpMem)) : nullptr;
    if (STENCIL) {
        const int w = 2 * A.kw.r + 1;
        for (int a = threadIdx.x; a < w * w * w; a += SW_THREADS) kt[a] = A.k3[a];
    }
    for (int a = threadIdx.x; a <= 2 * A.kw.r; a += SW_THREADS) S.qw[a] = A.kw.q[a];
    for (int a = threadIdx.x; a < kOwnWords; a += SW_THREADS) S.own[a] = 0u;
    if (threadIdx.x == 0) {
        S.abort_flag = 0;
        S.ncnt = 1u;
        S.nown = 0;
    }
    __syncthreads();
    unsigned target = 0;      // thread 0: arrivals the next barrier waits for
    double e_lane = 0.0;
    unsigned n_lane = 0;
    unsigned long long t_dec = 0, t_upd = 0;   // thread 0: tiles visited per phase
    int round = 0, capped = 0;
    bool marked = false;      // the last update stamped the tiles to decide
    // opening pass: leaders of the starting labels
    for (int base = 0; base < per_block; base += kListCap) {
        const int n = list_tiles(S, base, per_block, ntiles, [](int, int) { return true; });
        for (int q = wp; q < n; q += NWARP) {
            const int t = S.list[q];
            const bool now = tile_update<STENCIL>(A, M, S.qw, kt, t, true, -1);
            if (lane == 0) set_own(A, S, t, now);
        }
    }
    if (!grid_barrier(A.bar, A.err, A.spin_limit, target, &S.abort_flag)) return;
    for (int k = 0;; ++k) {
        if (k >= A.max_rounds) {     // cap reached: capped if leaders are left
            round = k;
            capped = -1;
            break;
        }
        // decide (the global leader count is read meanwhile; it only
        // changes in the update phases)
        unsigned nl = 1u;
        if (threadIdx.x == 0) nl = ld_relaxed_u32(A.nlead);
        const bool stamped = marked && (A.stamps > 0 || S.nown > NWARP);
        for (int base = 0; base < per_block; base += kListCap) {
            const int n = list_tiles(S, base, per_block, ntiles, [&](int j, int t) {
                return own_bit(S, j) && (!stamped || __ldcg(A.dirty + t) == k);
            });
            t_dec += (unsigned long long)n;
            for (int q = wp; q < n; q += NWARP) tile_decide(A, M, S.list[q], e_lane, n_lane);
        }
        if (threadIdx.x == 0) S.ncnt = nl;
        __syncthreads();
        if (S.ncnt == 0u) {          // no leader was left: converged
            round = k;
            break;
        }
        if (!grid_barrier(A.bar, A.err, A.spin_limit, target, &S.abort_flag)) return;
        // update (S.ncnt: the leader tiles of this round, alike in every block)
        marked = A.stamps > 0 || (A.stamps < 0 && S.ncnt > (unsigned)(NWARP * gridDim.x));
        const int mark = marked ? k + 1 : -1;
        for (int base = 0; base < per_block; base += kListCap) {
            const int n = list_tiles(S, base, per_block, ntiles, [&](int, int t) {
                const bool f = __ldcg(A.upd + t) != 0;
                if (f) A.upd[t] = 0;
                return f;
            });
            t_upd += (unsigned long long)n;
            for (int q = wp; q < n; q += NWARP) {
                const int t = S.list[q];
                const bool now = tile_update<STENCIL>(A, M, S.qw, kt, t, false, mark);
                if (lane == 0) set_own(A, S, t, now);
            }
        }
        if (!grid_barrier(A.bar, A.err, A.spin_limit, target, &S.abort_flag)) return;
    }
    // FP64 sums of the flipped cells' dE and their counts: lanes, then warps
    // in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e_lane += __shfl_down_sync(0xffffffffu, e_lane, o);
        n_lane += __shfl_down_sync(0xffffffffu, n_lane, o);
    }
    if (lane == 0) {
        S.e[wp] = e_lane;
        S.nf[wp] = n_lane;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double te = 0.0;
        unsigned long long tf = 0;
        for (int q = 0; q < NWARP; ++q) {
            te += S.e[q];
            tf += S.nf[q];
        }
        A.part_flips[blockIdx.x] = tf;
        A.part_dE[blockIdx.x] = te;
        A.part_tiles[blockIdx.x] = t_dec;
        A.part_tiles[gridDim.x + blockIdx.x] = t_upd;
        if (blockIdx.x == 0) {
            *A.rounds_out = round;
            *A.capped_out = capped < 0 ? (ld_relaxed_u32(A.nlead) != 0u) : 0;
        }
    }
}

__global__ void k_sweep_final(const unsigned long long *part_flips,
                              const double *part_dE, const unsigned long long *part_tiles,
                              int nb, const int *rounds, const int *capped, RoundState *rs)
{
    unsigned long long f = 0, td = 0, tu = 0;
    double e = 0.0;
    for (int b = 0; b < nb; ++b) {
        f += part_flips[b];
        e += part_dE[b];
        td += part_tiles[b];
        tu += part_tiles[nb + b];
    }
    rs->tiles_decide = td;
    rs->tiles_update = tu;
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

static size_t pad256(size_t x) { return (x + 255) / 256 * 256; }

// Sweep state: leader words, leader offsets, the per-tile posting areas,
// the update flags, the decide stamps and the label bits.
size_t sweep_state_bytes(const GridDesc &g, int r)
{
    const size_t nt = (size_t)sweep_tiles(g);
    const size_t nb = (size_t)sweep_bricks(g, r);
    const size_t nzw = ((size_t)g.nz + 31) / 32;
    return nb * 8 + pad256(nb) + nt * kPostBytes + pad256(nt) + pad256(nt * 4) +
           (size_t)g.nx * g.ny * nzw * 4;
}

// Label bits: word w of column (i, j) holds cells 32 w .. 32 w + 31 of the
// column (bit = cell - 32 w), zero past its end; the words are stored plane
// by plane, word (w, i, j) at (w nx + i) ny + j.
__global__ void k_pack_labels(const uint8_t *__restrict__ chi, int nz, long long nxy,
                              long long nwords, unsigned *__restrict__ CB)
{
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    const long long wz = w / nxy, col = w - wz * nxy;
    const int k0 = (int)wz * 32;
    const uint8_t *src = chi + col * nz + k0;
    const int n = min(32, nz - k0);
    unsigned b = 0u;
    if (n == 32 && ((uintptr_t)src & 15u) == 0) {   // two 16-byte loads
        const uint4 v0 = *reinterpret_cast<const uint4 *>(src);
        const uint4 v1 = *reinterpret_cast<const uint4 *>(src + 16);
        const unsigned q[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int k = 0; k < 32; ++k)
            b |= (((q[k >> 2] >> (8 * (k & 3))) & 0xffu) != 0u ? 1u : 0u) << k;
    } else {
        for (int k = 0; k < n; ++k) b |= (src[k] != 0 ? 1u : 0u) << k;
    }
    CB[w] = b;
}

// warps' areas plus room for the largest full stencil ((2 * 8 + 1)^3 ints)
constexpr size_t kSweepSmem =
    NWARP * sizeof(WarpMem) + sizeof(int) * (2 * kMaxR + 1) * (2 * kMaxR + 1) * (2 * kMaxR + 1);

cudaError_t sweep_grid_size(int nsm, int r, int *blocks)
{
    (void)r;
    cudaError_t e = cudaFuncSetAttribute(k_sweep<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSweepSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSweepSmem);
    if (e != cudaSuccess) return e;
    int per = 0, per2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<false>, SW_THREADS,
                                                      kSweepSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_sweep<true>, SW_THREADS,
                                                      kSweepSmem);
    if (e != cudaSuccess) return e;
    per = per2 < per ? per2 : per;
    per = per > VESIS_SWEEP_BPS ? VESIS_SWEEP_BPS : per;
    *blocks = per * nsm;
    return *blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

int sweep_ctl_words() { return 3 * kLine; }

// Arguments of one system's sweep, with its set-up enqueued on st: the
// posting bitmaps, update flags and control words cleared and the label
// bits packed (leader words are all rewritten by the opening pass).
static SweepArgs sweep_setup(const GridDesc &g, const KernelW &kw, const int *k3,
                             const FlipConst &fc, uint8_t *chi, uint32_t *W, const float *U,
                             double *dE, void *state, unsigned *ctl, int *err, int max_rounds,
                             long long spin_limit, cudaStream_t st)
{
    SweepArgs A;
    A.g = g;
    A.kw = kw;
    A.cD = fc.cN;
    A.h3 = fc.h3;
    A.qc3 = fc.k0;
    A.ksum = fc.S;
    A.k3 = k3;
    A.chi = chi;
    A.W = W;
    A.U = U;
    A.dE = dE;
    A.ntx = (g.nx + TS - 1) / TS;
    A.nty = (g.ny + TS - 1) / TS;
    A.ntz = (g.nz + TS - 1) / TS;
    A.bs = sweep_brick_edge(kw.r);
    A.bsh = A.bs == 4 ? 2 : 1;
    A.reach = (kw.r + A.bs - 1) / A.bs;
    A.nbx = (g.nx + A.bs - 1) / A.bs;
    A.nby = (g.ny + A.bs - 1) / A.bs;
    A.nbz = (g.nz + A.bs - 1) / A.bs;
    A.vec = (g.nz % TS == 0) && ((uintptr_t)W % 16 == 0) && ((uintptr_t)U % 16 == 0);
    const size_t nb = (size_t)A.nbx * A.nby * A.nbz;
    const size_t nt = (size_t)A.ntx * A.nty * A.ntz;
    uint8_t *base = static_cast<uint8_t *>(state);
    A.PL = reinterpret_cast<unsigned long long *>(base);
    A.PO = base + nb * 8;
    A.post = A.PO + pad256(nb);
    A.upd = A.post + nt * kPostBytes;
    A.dirty = reinterpret_cast<int *>(A.upd + pad256(nt));
    A.CB = reinterpret_cast<unsigned *>(A.upd + pad256(nt) + pad256(nt * 4));
    A.nzw = (g.nz + 31) / 32;
    A.nlead = ctl;
    A.bar = ctl + kLine;
    A.err = err;
    A.part_flips = nullptr;
    A.part_dE = nullptr;
    A.part_tiles = nullptr;
    A.rounds_out = nullptr;
    A.capped_out = nullptr;
    A.max_rounds = max_rounds;
    A.spin_limit = spin_limit;
    A.stamps = -1;
    A.rs = nullptr;
    A.tile_dE = nullptr;
    A.tile_nf = nullptr;
    // postings start empty (a slot is only read under its bitmap bit)
    cudaMemset2DAsync(A.post + kPostMaskOff, kPostBytes, 0, 32, nt, st);
    cudaMemsetAsync(A.upd, 0, nt, st);
    cudaMemsetAsync(A.dirty, 0, nt * 4, st);
    cudaMemsetAsync(ctl, 0, sweep_ctl_words() * sizeof(unsigned), st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    {
        const long long nwords = (long long)g.nx * g.ny * A.nzw;
        count_launch();
        k_pack_labels<<<(unsigned)((nwords + 255) / 256), 256, 0, st>>>(
            chi, g.nz, (long long)g.nx * g.ny, nwords, A.CB);
    }
    return A;
}

cudaError_t launch_sweep(const GridDesc &g, const KernelW &kw, const int *k3,
                         const FlipConst &fc,
                         uint8_t *chi, uint32_t *W, const float *U,
                         double *dE, void *state, unsigned *ctl, int *err,
                         unsigned long long *part_flips, double *part_dE,
                         unsigned long long *part_tiles,
                         int *rounds, int *capped, int max_rounds, int blocks,
                         long long spin_limit, int stamps, RoundState *rs, cudaStream_t st)
{
    {
        const size_t nt = (size_t)sweep_tiles(g);
        if ((nt + blocks - 1) / blocks > (size_t)kOwnWords * 32) return cudaErrorInvalidValue;
    }
    SweepArgs A = sweep_setup(g, kw, k3, fc, chi, W, U, dE, state, ctl, err, max_rounds,
                              spin_limit, st);
    A.part_flips = part_flips;
    A.part_dE = part_dE;
    A.part_tiles = part_tiles;
    A.rounds_out = rounds;
    A.capped_out = capped;
    A.stamps = stamps;
    void *args[] = {&A};
    count_launch();
    cudaError_t e = cudaLaunchCooperativeKernel(k3 ? (void *)k_sweep<true> : (void *)k_sweep<false>,
                                                dim3(blocks),
                                                dim3(SW_THREADS), args, kSweepSmem, st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_sweep_final<<<1, 1, 0, st>>>(part_flips, part_dE, part_tiles, blocks, rounds, capped, rs);
    return cudaGetLastError();
}


// ------------------------------------------------- many systems at once
// The same rounds for up to kMaxSweepSys systems in one cooperative launch:
// the systems' tiles are numbered one after another and dealt round-robin
// over the blocks, each round's decide and update phases serve the tiles of
// every system, and one grid barrier closes each phase for all of them.
// Every system's leaders, postings, labels and W live in its own state
// exactly as in the single-system sweep, so each system goes through the
// same rounds as alone.  A system whose leaders are gone contributes no
// tiles; the launch ends when no system has any.  The FP64 sum of a tile's
// flipped dE is kept per tile (the tile's warp adds it, round after round)
// and summed over the system's tiles in tile order at the end.

// dynamic shared memory offset of the systems' arguments (16-byte aligned)
constexpr size_t kSweepSysOff = (kSweepSmem + 15) / 16 * 16;

struct MultiArgs {
    const SweepArgs *sys;     // [nsys] (device)
    const long long *toff;    // [nsys + 1]: first global tile of each system
    int nsys;
    int ntiles;
    unsigned *nlead;          // tiles holding a leader, all systems (own line)
    unsigned *bar;            // grid barrier arrivals (own line)
    int *err;
    int *rounds;              // [nsys]
    int *capped;              // [nsys]
    int max_rounds;
    long long spin_limit;
    int stamps;               // as SweepArgs::stamps, for all systems
    KernelW kw;
    const int *k3;
};

__device__ __forceinline__ int sys_of(const long long *toff, int nsys, long long tg)
{
    int lo = 0, hi = nsys;    // toff[lo] <= tg < toff[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (toff[mid] <= tg) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The block's tiles that received a winner, over the global tile numbers,
// each flag read (and cleared) in its own system's update flags.
__device__ int gather_tiles_multi(SweepShared &S, const SweepArgs *sys, const long long *toff,
                                  int nsys, int base, int per_block, int ntiles)
{
    return list_tiles(S, base, per_block, ntiles, [&](int, int t) {
        const int q = sys_of(toff, nsys, t);
        uint8_t *f = sys[q].upd + (t - toff[q]);
        const bool fl = __ldcg(f) != 0;
        if (fl) *f = 0;
        return fl;
    });
}

__device__ __forceinline__ void set_own_multi(SweepShared &S, long long tg, bool now,
                                              unsigned *nlead_all, unsigned *nlead_sys)
{
    const int j = (int)((tg - (long long)blockIdx.x) / (long long)gridDim.x);
    const unsigned bit = 1u << (j & 31);
    const bool old = (S.own[j >> 5] & bit) != 0u;
    if (now == old) return;
    if (now) atomicOr(&S.own[j >> 5], bit);
    else atomicAnd(&S.own[j >> 5], ~bit);
    atomicAdd(&S.nown, now ? 1 : -1);
    red_add(nlead_all, now ? 1u : 0xffffffffu);
    red_add(nlead_sys, now ? 1u : 0xffffffffu);
}

template <bool STENCIL>
__global__ void __launch_bounds__(SW_THREADS, 1)
k_sweep_multi(MultiArgs P)
{
    __shared__ SweepShared S;
    __shared__ long long s_toff[kMaxSweepSys + 1];
    __shared__ int s_rounds[kMaxSweepSys];
    extern __shared__ __align__(16) unsigned char dyn[];
    WarpMem *WM = reinterpret_cast<WarpMem *>(dyn);
    // after the warps' areas and the stencil: the systems' arguments
    SweepArgs *s_sys = reinterpret_cast<SweepArgs *>(dyn + kSweepSysOff);
    const int ntiles = P.ntiles, nsys = P.nsys;
    const int per_block = (ntiles + gridDim.x - 1) / gridDim.x;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    WarpMem &M = WM[wp];
    int *kt = STENCIL ? reinterpret_cast<int *>(dyn + NWARP * sizeof(WarpMem)) : nullptr;
    if (STENCIL) {
        const int w = 2 * P.kw.r + 1;
        for (int a = threadIdx.x; a < w * w * w; a += SW_THREADS) kt[a] = P.k3[a];
    }
    {
        const int words = nsys * (int)(sizeof(SweepArgs) / 4);
        const unsigned *src = reinterpret_cast<const unsigned *>(P.sys);
        unsigned *dst = reinterpret_cast<unsigned *>(s_sys);
        for (int a = threadIdx.x; a < words; a += SW_THREADS) dst[a] = src[a];
    }
    for (int a = threadIdx.x; a <= 2 * P.kw.r; a += SW_THREADS) S.qw[a] = P.kw.q[a];
    for (int a = threadIdx.x; a < kOwnWords; a += SW_THREADS) S.own[a] = 0u;
    for (int a = threadIdx.x; a <= nsys; a += SW_THREADS) s_toff[a] = P.toff[a];
    for (int a = threadIdx.x; a < nsys; a += SW_THREADS) s_rounds[a] = 0;
    if (threadIdx.x == 0) {
        S.abort_flag = 0;
        S.ncnt = 1u;
        S.nown = 0;
    }
    __syncthreads();
    unsigned target = 0;
    int capped = 0;
    bool marked = false;
    // opening pass: leaders of every system's starting labels
    for (int base = 0; base < per_block; base += kListCap) {
        const int n = list_tiles(S, base, per_block, ntiles, [](int, int) { return true; });
        for (int q = wp; q < n; q += NWARP) {
            const int tg = S.list[q];
            const int sq = sys_of(s_toff, nsys, tg);
            const SweepArgs &A = s_sys[sq];
            const bool now =
                tile_update<STENCIL>(A, M, S.qw, kt, (int)(tg - s_toff[sq]), true, -1);
            if (lane == 0) set_own_multi(S, tg, now, P.nlead, A.nlead);
        }
    }
    if (!grid_barrier(P.bar, P.err, P.spin_limit, target, &S.abort_flag)) return;
    for (int k = 0;; ++k) {
        if (k >= P.max_rounds) {
            capped = 1;
            break;
        }
        unsigned nl = 1u;
        if (threadIdx.x == 0) nl = ld_relaxed_u32(P.nlead);
        if (blockIdx.x == 0)         // rounds of each system that still had leaders
            for (int q = threadIdx.x; q < nsys; q += SW_THREADS)
                if (ld_relaxed_u32(s_sys[q].nlead) != 0u) s_rounds[q] = k + 1;
        const bool stamped = marked && (P.stamps > 0 || S.nown > NWARP);
        for (int base = 0; base < per_block; base += kListCap) {
            const int n = list_tiles(S, base, per_block, ntiles, [&](int j, int tg) {
                if (!own_bit(S, j)) return false;
                if (!stamped) return true;
                const int sq = sys_of(s_toff, nsys, tg);
                return __ldcg(s_sys[sq].dirty + (tg - s_toff[sq])) == k;
            });
            for (int q = wp; q < n; q += NWARP) {
                const int tg = S.list[q];
                const int sq = sys_of(s_toff, nsys, tg);
                const SweepArgs &A = s_sys[sq];
                const int t = (int)(tg - s_toff[sq]);
                double e = 0.0;
                unsigned nf = 0;
                tile_decide(A, M, t, e, nf);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    e += __shfl_down_sync(0xffffffffu, e, o);
                    nf += __shfl_down_sync(0xffffffffu, nf, o);
                }
                if (lane == 0 && nf) {
                    A.tile_dE[t] += e;
                    A.tile_nf[t] += nf;
                }
            }
        }
        if (threadIdx.x == 0) S.ncnt = nl;
        __syncthreads();
        if (S.ncnt == 0u) break;
        if (!grid_barrier(P.bar, P.err, P.spin_limit, target, &S.abort_flag)) return;
        marked = P.stamps > 0 || (P.stamps < 0 && S.ncnt > (unsigned)(NWARP * gridDim.x));
        const int mark = marked ? k + 1 : -1;
        for (int base = 0; base < per_block; base += kListCap) {
            const int n = gather_tiles_multi(S, s_sys, s_toff, nsys, base, per_block, ntiles);
            for (int q = wp; q < n; q += NWARP) {
                const int tg = S.list[q];
                const int sq = sys_of(s_toff, nsys, tg);
                const SweepArgs &A = s_sys[sq];
                const bool now =
                    tile_update<STENCIL>(A, M, S.qw, kt, (int)(tg - s_toff[sq]), false, mark);
                if (lane == 0) set_own_multi(S, tg, now, P.nlead, A.nlead);
            }
        }
        if (!grid_barrier(P.bar, P.err, P.spin_limit, target, &S.abort_flag)) return;
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        for (int q = threadIdx.x; q < nsys; q += SW_THREADS) {
            P.rounds[q] = s_rounds[q];
            P.capped[q] = capped && ld_relaxed_u32(s_sys[q].nlead) != 0u;
        }
    }
}

// Totals of system blockIdx.x: its tiles' flip counts and dE sums added in
// a fixed order (strided per thread, then a tree over the threads).
__global__ void __launch_bounds__(256) k_sweep_multi_final(const SweepArgs *sys,
                                                           const int *rounds, const int *capped)
{
    __shared__ double se[256];
    __shared__ unsigned long long sf[256];
    const SweepArgs &A = sys[blockIdx.x];
    const int nt = A.ntx * A.nty * A.ntz;
    double e = 0.0;
    unsigned long long f = 0;
    for (int t = threadIdx.x; t < nt; t += 256) {
        e += A.tile_dE[t];
        f += A.tile_nf[t];
    }
    se[threadIdx.x] = e;
    sf[threadIdx.x] = f;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            se[threadIdx.x] += se[threadIdx.x + w];
            sf[threadIdx.x] += sf[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        RoundState *rs = A.rs;
        rs->done = 1;
        rs->round = rounds[blockIdx.x];
        rs->capped = capped[blockIdx.x];
        rs->round_flips = 0;
        rs->total_flips = sf[0];
        rs->round_dE = 0.0;
        rs->total_dE = se[0];
        rs->tiles_decide = 0;
        rs->tiles_update = 0;
    }
}

static size_t pad256z(size_t x) { return (x + 255) / 256 * 256; }

size_t sweep_multi_scratch_bytes(int nsys)
{
    return pad256z((size_t)nsys * sizeof(SweepArgs)) + pad256z((size_t)(nsys + 1) * 8) +
           pad256z(3 * kLine * sizeof(unsigned)) + pad256z(sizeof(int)) +
           2 * pad256z((size_t)nsys * sizeof(int));
}

cudaError_t launch_sweep_multi(int nsys, const SweepSys *sys, const KernelW &kw, const int *k3,
                               int max_rounds, int blocks, long long spin_limit, int stamps,
                               void *scratch, int *err_out, cudaStream_t st)
{
    if (nsys < 1 || nsys > kMaxSweepSys) return cudaErrorInvalidValue;
    std::vector<SweepArgs> As((size_t)nsys);
    std::vector<long long> toff((size_t)nsys + 1, 0);
    for (int q = 0; q < nsys; ++q) {
        const SweepSys &y = sys[q];
        const int nt = sweep_tiles(y.g);
        toff[q + 1] = toff[q] + nt;
        As[q] = sweep_setup(y.g, kw, k3, y.fc, y.chi, y.W, y.U, y.dE, y.state, y.ctl, y.err,
                            max_rounds, spin_limit, y.st);
        As[q].rs = y.rs;
        As[q].tile_dE = y.tile_dE;
        As[q].tile_nf = y.tile_nf;
        cudaMemsetAsync(y.tile_dE, 0, (size_t)nt * sizeof(double), y.st);
        cudaMemsetAsync(y.tile_nf, 0, (size_t)nt * sizeof(unsigned), y.st);
    }
    if (toff[nsys] > 0x7fffffffll ||
        (toff[nsys] + blocks - 1) / blocks > (long long)kOwnWords * 32)
        return cudaErrorInvalidValue;
    // the systems' set-up ran on their own streams: st waits for all of it
    for (int q = 0; q < nsys; ++q) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        cudaEventRecord(ev, sys[q].st);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
    }
    uint8_t *b = static_cast<uint8_t *>(scratch);
    SweepArgs *d_sys = reinterpret_cast<SweepArgs *>(b);
    b += pad256z((size_t)nsys * sizeof(SweepArgs));
    long long *d_toff = reinterpret_cast<long long *>(b);
    b += pad256z((size_t)(nsys + 1) * 8);
    unsigned *d_ctl = reinterpret_cast<unsigned *>(b);
    b += pad256z(3 * kLine * sizeof(unsigned));
    int *d_err = reinterpret_cast<int *>(b);
    b += pad256z(sizeof(int));
    int *d_rounds = reinterpret_cast<int *>(b);
    b += pad256z((size_t)nsys * sizeof(int));
    int *d_capped = reinterpret_cast<int *>(b);
    cudaMemcpyAsync(d_sys, As.data(), (size_t)nsys * sizeof(SweepArgs), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_toff, toff.data(), (size_t)(nsys + 1) * 8, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(d_ctl, 0, 3 * kLine * sizeof(unsigned), st);
    cudaMemsetAsync(d_err, 0, sizeof(int), st);
    MultiArgs P;
    P.sys = d_sys;
    P.toff = d_toff;
    P.nsys = nsys;
    P.ntiles = (int)toff[nsys];
    P.nlead = d_ctl;
    P.bar = d_ctl + kLine;
    P.err = d_err;
    P.rounds = d_rounds;
    P.capped = d_capped;
    P.max_rounds = max_rounds;
    P.spin_limit = spin_limit;
    P.stamps = stamps;
    P.kw = kw;
    P.k3 = k3;
    const size_t smem = kSweepSysOff + (size_t)nsys * sizeof(SweepArgs);
    void *fn = k3 ? (void *)k_sweep_multi<true> : (void *)k_sweep_multi<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSweepSysOff + kMaxSweepSys * sizeof(SweepArgs)));
    if (e != cudaSuccess) return e;
    void *args[] = {&P};
    count_launch();
    e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(SW_THREADS), args, smem, st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_sweep_multi_final<<<nsys, 256, 0, st>>>(d_sys, d_rounds, d_capped);
    if (err_out) cudaMemcpyAsync(err_out, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    return cudaGetLastError();
}

}  // namespace vesis
