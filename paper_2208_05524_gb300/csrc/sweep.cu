// Persistent narrow-band flip sweep (Sec. 3.1, Step 2) for sm_103a.
//
// All flip rounds of one interface relaxation run in a single cooperative
// launch.  The grid is cut into 8^3 tiles; only tiles holding candidate
// cells (a face neighbour with the other label) are active, which is the
// band around the interface the paper restricts the flips to.  Per round:
//
//   phase A (active tiles): dE = c [s (1 - 2w) - g0] - s h^3 U in FP64 for
//     candidates (Eq. dGj1/dGj2), key = (ordered bits of float(dE)) << 32 |
//     index where dE < 0, else ~0; a tile without candidates turns inactive.
//   barrier
//   phase B (tiles with a negative candidate): load the keys of the tile and
//     a halo of r cells into shared memory, take the minimum over the cube
//     of half-width r by three separable passes, flip the cells whose key is
//     that minimum, add +-q_a q_b q_c to W over each flipped cell's window
//     with integer atomics (W stays the exact convolution), and activate the
//     tiles of the flipped cells and of their face neighbours.
//   barrier; stop when the round flipped nothing.
//
// Selected cells are more than r apart, so they do not interact through the
// kernel and the round lowers the energy by exactly the sum of their dE.
// The grid barrier spins with a bound; on timeout it raises an error flag
// and every block returns.
#include <cooperative_groups.h>

#include "vesis_internal.cuh"

namespace vesis {

constexpr int TS = 8;             // tile edge
constexpr int TC = TS * TS * TS;  // cells per tile
constexpr int SW_THREADS = 256;
constexpr long long kSpinLimit = 1ll << 26;

struct SweepArgs {
    GridDesc g;
    KernelW kw;
    FlipConst fc;
    uint8_t *chi;
    uint32_t *W;
    const float *U;
    unsigned long long *K;
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
};

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
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)A.err == 0;
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

__device__ __forceinline__ unsigned long long flip_key_s(double dE, long long p)
{
    unsigned u = __float_as_uint(__double2float_rn(dE));
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (unsigned long long)p;
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

// Phase A for one tile: keys and flip energies of its cells.
__device__ void phase_keys(const SweepArgs &A, int t, uint8_t *act_next)
{
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    bool cand_any = false, neg_any = false;
#pragma unroll
    for (int u = 0; u < TC / SW_THREADS; ++u) {
        const int c = threadIdx.x + u * SW_THREADS;
        const int i = i0 + c / (TS * TS), j = j0 + (c / TS) % TS, k = k0 + c % TS;
        if (i >= g.nx || j >= g.ny || k >= g.nz) continue;
        const long long p = (long long)i * nyz + (long long)j * g.nz + k;
        // labels, W and keys change under other blocks between rounds:
        // read them at L2 (ld.global.cg), never from a stale L1 line
        const uint8_t x = __ldcg(A.chi + p);
        const uint8_t xm = (i > 0) ? __ldcg(A.chi + p - nyz) : 0;
        const uint8_t xp = (i < g.nx - 1) ? __ldcg(A.chi + p + nyz) : 0;
        const uint8_t ym = (j > 0) ? __ldcg(A.chi + p - g.nz) : 0;
        const uint8_t yp = (j < g.ny - 1) ? __ldcg(A.chi + p + g.nz) : 0;
        const uint8_t zm = (k > 0) ? __ldcg(A.chi + p - 1) : 0;
        const uint8_t zp = (k < g.nz - 1) ? __ldcg(A.chi + p + 1) : 0;
        const bool cand = (xm != x) | (xp != x) | (ym != x) | (yp != x) |
                          (zm != x) | (zp != x);
        unsigned long long key = ~0ull;
        if (cand) {
            cand_any = true;
            const double e = flip_dE_s(x, __ldcg(A.W + p), __ldg(A.U + p), A.fc);
            if (e < 0.0) {
                A.dE[p] = e;
                key = flip_key_s(e, p);
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

// Phase B for one tile: window minimum, flips, W update, activation.
__device__ void phase_flip(const SweepArgs &A, int t, uint8_t *act_next,
                           unsigned long long *smem, unsigned &nflip,
                           double &esum)
{
    __shared__ int s_nf;
    __shared__ long long s_fl[TC];
    const int r = A.kw.r;
    const int H = TS + 2 * r;
    const int w = 2 * r + 1;
    unsigned long long *Kh = smem;                     // H^3, later M2
    unsigned long long *M1 = smem + H * H * H;         // H * H * TS
    int i0, j0, k0;
    tile_origin(A, t, i0, j0, k0);
    const GridDesc &g = A.g;
    const long long nyz = (long long)g.ny * g.nz;
    if (threadIdx.x == 0) s_nf = 0;
    for (int idx = threadIdx.x; idx < H * H * H; idx += SW_THREADS) {
        const int hz = idx % H, hy = (idx / H) % H, hx = idx / (H * H);
        const int i = i0 - r + hx, j = j0 - r + hy, k = k0 - r + hz;
        unsigned long long v = ~0ull;
        if (i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz)
            v = __ldcg(A.K + (long long)i * nyz + (long long)j * g.nz + k);
        Kh[idx] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < H * H * TS; idx += SW_THREADS) {
        const int z = idx % TS, hy = (idx / TS) % H, hx = idx / (TS * H);
        const unsigned long long *col = Kh + (hx * H + hy) * H + z;
        unsigned long long m = col[0];
        for (int d = 1; d < w; ++d) m = min(m, col[d]);
        M1[idx] = m;
    }
    unsigned long long key[TC / SW_THREADS];
#pragma unroll
    for (int u = 0; u < TC / SW_THREADS; ++u) {
        const int c = threadIdx.x + u * SW_THREADS;
        const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
        key[u] = Kh[((x + r) * H + (y + r)) * H + (z + r)];
    }
    __syncthreads();
    unsigned long long *M2 = Kh;                       // H * TS * TS
    for (int idx = threadIdx.x; idx < H * TS * TS; idx += SW_THREADS) {
        const int z = idx % TS, y = (idx / TS) % TS, hx = idx / (TS * TS);
        const unsigned long long *col = M1 + (hx * H + y) * TS + z;
        unsigned long long m = col[0];
        for (int d = 1; d < w; ++d) m = min(m, col[d * TS]);
        M2[idx] = m;
    }
    __syncthreads();
    double e = 0.0;
#pragma unroll
    for (int u = 0; u < TC / SW_THREADS; ++u) {
        const int c = threadIdx.x + u * SW_THREADS;
        if (key[u] == ~0ull) continue;
        const int x = c / (TS * TS), y = (c / TS) % TS, z = c % TS;
        const unsigned long long *col = M2 + (x * TS + y) * TS + z;
        unsigned long long m = col[0];
        for (int d = 1; d < w; ++d) m = min(m, col[d * TS * TS]);
        if (m == key[u]) {
            const long long p = (long long)(key[u] & 0xffffffffull);
            A.chi[p] = (uint8_t)(1 - __ldcg(A.chi + p));
            e += __ldcg(A.dE + p);
            const int slot = atomicAdd(&s_nf, 1);
            s_fl[slot] = p;
        }
    }
    // fixed-order block sum of the flipped cells' dE (each cell's dE sits
    // in a fixed thread and slot, so the order does not depend on timing)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    __shared__ double s_e[SW_THREADS / 32];
    if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = e;
    __syncthreads();
    const int nf = s_nf;
    if (threadIdx.x == 0) {
        double te = 0.0;
        for (int q = 0; q < SW_THREADS / 32; ++q) te += s_e[q];
        esum += te;
        nflip += (unsigned)nf;
    }
    // W update and activation for each flipped cell
    for (int f = 0; f < nf; ++f) {
        const long long p = s_fl[f];
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
}

__global__ void __launch_bounds__(SW_THREADS)
k_sweep(SweepArgs A)
{
    extern __shared__ unsigned long long smem[];
    const int ntiles = A.ntx * A.nty * A.ntz;
    unsigned nflip = 0;       // thread 0 only
    double esum = 0.0;        // thread 0 only
    int round = 0, capped = 0;
    for (;;) {
        uint8_t *cur = (round & 1) ? A.act1 : A.act0;
        uint8_t *nxt = (round & 1) ? A.act0 : A.act1;
        if (blockIdx.x == 0 && threadIdx.x == 0) A.cnt[(round + 1) % 3] = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (__ldcg(cur + t)) {
                phase_keys(A, t, nxt);
            } else if (threadIdx.x == 0) {
                nxt[t] = 0;
                A.tneg[t] = 0;
            }
        }
        if (!grid_barrier(A)) return;
        const unsigned before = nflip;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            if (__ldcg(A.tneg + t)) phase_flip(A, t, nxt, smem, nflip, esum);
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
    const int H = TS + 2 * r;
    return sizeof(unsigned long long) * ((size_t)H * H * H + (size_t)H * H * TS);
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
    *blocks = per * nsm;
    return *blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t launch_sweep(const GridDesc &g, const KernelW &kw, const FlipConst &fc,
                         uint8_t *chi, uint32_t *W, const float *U,
                         unsigned long long *K, double *dE, uint8_t *act,
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
    // every tile starts active: round 0 is a full pass that finds the band
    cudaMemsetAsync(act, 1, ntiles, st);
    cudaMemsetAsync(act + ntiles, 0, ntiles, st);
    cudaMemsetAsync(ctl, 0, 5 * sizeof(unsigned), st);
    cudaMemsetAsync(err, 0, sizeof(int), st);
    void *args[] = {&A};
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
