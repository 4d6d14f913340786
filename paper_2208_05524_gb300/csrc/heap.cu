// The paper's literal flipping process (Sec. 3.1, Steps 2.1-2.2): keep the
// flip candidates with dE < 0 in a min-heap ordered by (dE, linear index),
// flip the top, update w and dE in the kernel window of the flipped cell and
// the candidate set, and repeat until no candidate lowers the energy.
//
// The heap's valid entries are always exactly the current candidates with
// dE < 0 at their current dE (a cell's dE and its candidacy only change when
// a cell of its window flips), so the top is the smallest (dE, index) over
// the grid.  Here that minimum is kept in a two-level tournament instead of
// a pointer heap: the best key of every 4^3 tile and of every 8^3 group of
// tiles.  A flip rewrites the keys of its window, the tiles that cover the
// window and their groups; the next top is the best of the groups.  One
// block of 1024 threads runs the whole process, so it needs no grid
// barrier; the flips are as serial as the paper's.
//
// A cell's key is the bit pattern of its FP64 dE when dE < 0 (for negative
// doubles a larger pattern is a more negative value, so the order of the
// keys as unsigned integers is the reverse of the order of dE) and 0 for a
// cell that is not a candidate or has dE >= 0; ties go to the smaller
// linear index.  Comparisons are integer; the flipped cells' dE are summed
// in flip order in FP64.
#include "vesis_internal.cuh"

namespace vesis {

constexpr int HT = 4;        // tile edge (64 cells)
constexpr int HG = 8;        // tiles per group edge
constexpr int HB = 1024;     // threads of the flipping block
constexpr int HW = HB / 32;

typedef unsigned long long hkey;

// (e1, i1) comes before (e2, i2) in the heap's order
__device__ __forceinline__ bool key_less(hkey e1, int i1, hkey e2, int i2)
{
    return e1 > e2 || (e1 == e2 && i1 < i2);
}

__device__ __forceinline__ void warp_best(hkey &e, int &i)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const hkey e2 = __shfl_down_sync(0xffffffffu, e, o);
        const int i2 = __shfl_down_sync(0xffffffffu, i, o);
        if (key_less(e2, i2, e, i)) {
            e = e2;
            i = i2;
        }
    }
}

struct HeapArgs {
    GridDesc g;
    KernelW kw;
    const int *k3;        // full stencil or NULL (separable q)
    FlipConst fc;
    uint8_t *chi;
    uint32_t *W;
    const float *U;
    hkey *key;            // per cell
    hkey *te;             // per tile
    int *ti;
    hkey *ge;             // per group
    int *gi;
    int ntx, nty, ntz;    // tiles per axis
    int ngx, ngy, ngz;    // groups per axis
    long long max_flips;
    long long *flips_out;
    double *dsum_out;
    int *capped_out;
};

// The labels change inside k_heap_run, so they are read with plain loads
// (the read-only path of a const __restrict__ pointer is not coherent with
// the block's own stores).
__device__ __forceinline__ bool candidate_rw(const GridDesc &g, const uint8_t *chi, long long p,
                                             int i, int j, int k, long long nyz)
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

__device__ __forceinline__ hkey cell_key(const HeapArgs &A, long long p, int i, int j, int k,
                                         long long nyz)
{
    if (!candidate_rw(A.g, A.chi, p, i, j, k, nyz)) return 0ull;
    const double e = flip_dE(A.chi[p], A.W[p], A.U[p], A.fc);
    return e < 0.0 ? (hkey)__double_as_longlong(e) : 0ull;
}

// Best key of tile t (one warp; two cells per lane).
__device__ __forceinline__ void tile_best(const HeapArgs &A, int t, int lane, long long nyz)
{
    const int tz = t % A.ntz, ty = (t / A.ntz) % A.nty, tx = t / (A.ntz * A.nty);
    hkey e = 0ull;
    int idx = 0x7fffffff;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        const int i = tx * HT + (c >> 4), j = ty * HT + ((c >> 2) & 3), k = tz * HT + (c & 3);
        if (i < A.g.nx && j < A.g.ny && k < A.g.nz) {
            const long long p = (long long)i * nyz + (long long)j * A.g.nz + k;
            const hkey v = A.key[p];
            if (key_less(v, (int)p, e, idx)) {
                e = v;
                idx = (int)p;
            }
        }
    }
    warp_best(e, idx);
    if (lane == 0) {
        A.te[t] = e;
        A.ti[t] = idx;
    }
}

// Best key of group q (one warp over its up to 512 tiles).
__device__ __forceinline__ void group_best(const HeapArgs &A, int q, int lane)
{
    const int gz = q % A.ngz, gy = (q / A.ngz) % A.ngy, gx = q / (A.ngz * A.ngy);
    hkey e = 0ull;
    int idx = 0x7fffffff;
    for (int c = lane; c < HG * HG * HG; c += 32) {
        const int tx = gx * HG + c / (HG * HG), ty = gy * HG + (c / HG) % HG, tz = gz * HG + c % HG;
        if (tx < A.ntx && ty < A.nty && tz < A.ntz) {
            const int t = (tx * A.nty + ty) * A.ntz + tz;
            const hkey v = A.te[t];
            const int vi = A.ti[t];
            if (key_less(v, vi, e, idx)) {
                e = v;
                idx = vi;
            }
        }
    }
    warp_best(e, idx);
    if (lane == 0) {
        A.ge[q] = e;
        A.gi[q] = idx;
    }
}

__global__ void k_heap_keys(HeapArgs A)
{
    const long long nyz = (long long)A.g.ny * A.g.nz;
    const long long G = nyz * A.g.nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= G) return;
    const int i = (int)(p / nyz);
    const long long rem = p - (long long)i * nyz;
    const int j = (int)(rem / A.g.nz);
    const int k = (int)(rem - (long long)j * A.g.nz);
    A.key[p] = cell_key(A, p, i, j, k, nyz);
}

__global__ void k_heap_tiles(HeapArgs A, int ntiles)
{
    const int t = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (t >= ntiles) return;
    tile_best(A, t, threadIdx.x & 31, (long long)A.g.ny * A.g.nz);
}

__global__ void k_heap_groups(HeapArgs A, int ngroups)
{
    const int q = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (q >= ngroups) return;
    group_best(A, q, threadIdx.x & 31);
}

__global__ void __launch_bounds__(HB, 1) k_heap_run(HeapArgs A)
{
    __shared__ hkey s_e[HW];
    __shared__ int s_i[HW];
    __shared__ int s_q[7];     // top cell (index, i, j, k), sign, stop
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long nyz = (long long)A.g.ny * A.g.nz;
    const int ngroups = A.ngx * A.ngy * A.ngz;
    const int r = A.kw.r, wd = 2 * r + 1;
    long long flips = 0;
    double dsum = 0.0;
    int capped = 0;
    for (;;) {
        // top of the heap: best over the groups
        hkey e = 0ull;
        int idx = 0x7fffffff;
        for (int q = threadIdx.x; q < ngroups; q += HB) {
            const hkey v = A.ge[q];
            const int vi = A.gi[q];
            if (key_less(v, vi, e, idx)) {
                e = v;
                idx = vi;
            }
        }
        warp_best(e, idx);
        if (lane == 0) {
            s_e[wp] = e;
            s_i[wp] = idx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < HW; ++w)
                if (key_less(s_e[w], s_i[w], e, idx)) {
                    e = s_e[w];
                    idx = s_i[w];
                }
            int stop = 0;
            if (e == 0ull) {
                stop = 1;                       // no candidate lowers the energy
            } else if (flips >= A.max_flips) {
                stop = 1;
                capped = 1;
            } else {
                const long long p = idx;
                s_q[0] = idx;
                s_q[1] = (int)(p / nyz);
                s_q[2] = (int)((p / A.g.nz) % A.g.ny);
                s_q[3] = (int)(p % A.g.nz);
                s_q[4] = A.chi[p] ? -1 : 1;     // +1: solvent -> solute
                A.chi[p] ^= 1;
                ++flips;
                dsum += __longlong_as_double((long long)e);
            }
            s_q[5] = stop;
        }
        __syncthreads();
        if (s_q[5]) break;
        const int pi = s_q[1], pj = s_q[2], pk = s_q[3], sgn = s_q[4];
        // window: w of every cell, then its key (only the top changed label)
        const int nw = wd * wd * wd;
        for (int c = threadIdx.x; c < nw; c += HB) {
            const int a = c / (wd * wd) - r, b = (c / wd) % wd - r, d = c % wd - r;
            const int i = pi + a, j = pj + b, k = pk + d;
            if (i < 0 || i >= A.g.nx || j < 0 || j >= A.g.ny || k < 0 || k >= A.g.nz) continue;
            const long long p = (long long)i * nyz + (long long)j * A.g.nz + k;
            const int kwt = A.k3 ? A.k3[c] : A.kw.q[a + r] * A.kw.q[b + r] * A.kw.q[d + r];
            A.W[p] += (unsigned)(sgn * kwt);
            A.key[p] = cell_key(A, p, i, j, k, nyz);
        }
        __syncthreads();
        // tiles covering the window
        const int tx0 = max(pi - r, 0) / HT, tx1 = min(pi + r, A.g.nx - 1) / HT;
        const int ty0 = max(pj - r, 0) / HT, ty1 = min(pj + r, A.g.ny - 1) / HT;
        const int tz0 = max(pk - r, 0) / HT, tz1 = min(pk + r, A.g.nz - 1) / HT;
        const int mx = tx1 - tx0 + 1, my = ty1 - ty0 + 1, mz = tz1 - tz0 + 1;
        for (int c = wp; c < mx * my * mz; c += HW) {
            const int t = ((tx0 + c / (my * mz)) * A.nty + ty0 + (c / mz) % my) * A.ntz +
                          tz0 + c % mz;
            tile_best(A, t, lane, nyz);
        }
        __syncthreads();
        // their groups
        const int gx0 = tx0 / HG, gx1 = tx1 / HG, gy0 = ty0 / HG, gy1 = ty1 / HG;
        const int gz0 = tz0 / HG, gz1 = tz1 / HG;
        const int ux = gx1 - gx0 + 1, uy = gy1 - gy0 + 1, uz = gz1 - gz0 + 1;
        for (int c = wp; c < ux * uy * uz; c += HW) {
            const int q = ((gx0 + c / (uy * uz)) * A.ngy + gy0 + (c / uz) % uy) * A.ngz +
                          gz0 + c % uz;
            group_best(A, q, lane);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *A.flips_out = flips;
        *A.dsum_out = dsum;
        *A.capped_out = capped;
    }
}

size_t heap_state_bytes(const GridDesc &g)
{
    const size_t nt = (size_t)((g.nx + HT - 1) / HT) * ((g.ny + HT - 1) / HT) *
                      ((g.nz + HT - 1) / HT);
    const int tx = (g.nx + HT - 1) / HT, ty = (g.ny + HT - 1) / HT, tz = (g.nz + HT - 1) / HT;
    const size_t ng = (size_t)((tx + HG - 1) / HG) * ((ty + HG - 1) / HG) * ((tz + HG - 1) / HG);
    return (nt + ng) * (sizeof(hkey) + sizeof(int)) + 256;
}

cudaError_t launch_heap(const GridDesc &g, const KernelW &kw, const int *k3,
                        const FlipConst &fc, uint8_t *chi, uint32_t *W, const float *U,
                        double *key, void *state, long long max_flips, long long *flips_out,
                        double *dsum_out, int *capped_out, cudaStream_t st)
{
    HeapArgs A;
    A.g = g;
    A.kw = kw;
    A.k3 = k3;
    A.fc = fc;
    A.chi = chi;
    A.W = W;
    A.U = U;
    A.key = reinterpret_cast<hkey *>(key);
    A.ntx = (g.nx + HT - 1) / HT;
    A.nty = (g.ny + HT - 1) / HT;
    A.ntz = (g.nz + HT - 1) / HT;
    A.ngx = (A.ntx + HG - 1) / HG;
    A.ngy = (A.nty + HG - 1) / HG;
    A.ngz = (A.ntz + HG - 1) / HG;
    const long long nt = (long long)A.ntx * A.nty * A.ntz;
    const long long ng = (long long)A.ngx * A.ngy * A.ngz;
    uint8_t *base = static_cast<uint8_t *>(state);
    A.te = reinterpret_cast<hkey *>(base);
    A.ge = A.te + nt;
    A.ti = reinterpret_cast<int *>(A.ge + ng);
    A.gi = A.ti + nt;
    A.max_flips = max_flips;
    A.flips_out = flips_out;
    A.dsum_out = dsum_out;
    A.capped_out = capped_out;
    const long long G = (long long)g.nx * g.ny * g.nz;
    count_launch(4);
    k_heap_keys<<<(unsigned)((G + 255) / 256), 256, 0, st>>>(A);
    k_heap_tiles<<<(unsigned)((nt * 32 + 255) / 256), 256, 0, st>>>(A, (int)nt);
    k_heap_groups<<<(unsigned)((ng * 32 + 255) / 256), 256, 0, st>>>(A, (int)ng);
    k_heap_run<<<1, HB, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace vesis
