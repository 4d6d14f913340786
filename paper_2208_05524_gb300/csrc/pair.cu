// Grid x atom pair kernels of the VESIS hot path (sm_103a, FP32 CUDA cores).
//
// Energy density (Eq. Ur): U(x) = rho_w sum_i U_LJ^(i)(r) + C |E(x)|^2 with
// E(x) = sum_i Q_i d / r^3, d = x - r_i, r = max(|d|, r_min).  U_LJ is
// written A r^-12 - B r^-6 with A = 4 eps sigma^12, B = 4 eps sigma^6.
//
// Gradient (exact derivative of the discrete energy, Eq. GradientG):
//   d/dr_n [rho_w U_LJ] = rho_w r^-8 (12 A r^-6 - 6 B) d
//   d/dr_n [C |E|^2]    = -2 C Q_n [E r^-3 - 3 (d.E) d r^-5]
// with the LJ part and the d d^T part dropped where r is clamped.
//
// Atom tiles are staged in shared memory and read as warp-wide broadcasts;
// every thread keeps 4 or 8 cells of one z-pencil in registers, so the x/y
// parts of the distance are formed once per atom and reused.
#include "vesis_internal.cuh"

namespace vesis {

constexpr int PE_THREADS = 128;
constexpr int PE_TILE = 256;

// 1/sqrt(x) on the SFU without the subnormal range handling: every argument
// here is at least r_min^2, so flushing subnormals changes nothing.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two FP32 values in one 64-bit register, for the packed f32x2 arithmetic
// of sm_100-class SMs: one instruction performs the same IEEE operation on
// both halves, so the FP32 pipe is fed with half the issue slots.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void upk2(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Block-wide min and max of three values (all threads must call).
__device__ __forceinline__ void block_box(float x, float y, float z, float lo[3],
                                          float hi[3], float *s_box)
{
    float v[6] = {x, y, z, -x, -y, -z};
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] = fminf(v[c], __shfl_xor_sync(0xffffffffu, v[c], o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) s_box[w * 6 + c] = v[c];
    __syncthreads();
    float r[6] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f};
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
#pragma unroll
        for (int c = 0; c < 6; ++c) r[c] = fminf(r[c], s_box[q * 6 + c]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = r[c];
        hi[c] = -r[c + 3];
    }
}

// One staged atom, every value duplicated into both halves of a pair.
struct AtomPairs {
    f2 x, y, z, q;   // position, charge
    f2 a, nb;        // A = 4 eps sigma^12, -B = -4 eps sigma^6
};

// One atom against the PTS cells of a thread, two cells per packed
// instruction; CLAMP applies r_min.
template <bool CLAMP, int PTS>
__device__ __forceinline__ void energy_atom(const AtomPairs &at, f2 px, f2 py, const f2 *pz,
                                            float rmin2, f2 *lj, f2 *ex, f2 *ey, f2 *ez)
{
    const f2 dx = sub2(px, at.x);
    const f2 dy = sub2(py, at.y);
    const f2 dxy2 = fma2(dx, dx, mul2(dy, dy));
#pragma unroll
    for (int p = 0; p < PTS / 2; ++p) {
        const f2 dz = sub2(pz[p], at.z);
        const f2 r2 = fma2(dz, dz, dxy2);
        float r2a, r2b;
        upk2(r2, r2a, r2b);
        if (CLAMP) {
            r2a = fmaxf(r2a, rmin2);
            r2b = fmaxf(r2b, rmin2);
        }
        const f2 ri = pk2(rsqrt_ftz(r2a), rsqrt_ftz(r2b));
        const f2 ri2 = mul2(ri, ri);
        const f2 ri3 = mul2(ri2, ri);
        const f2 ri6 = mul2(ri3, ri3);
        const f2 tl = fma2(at.a, ri6, at.nb);    // A r^-6 - B
        lj[p] = fma2(ri6, tl, lj[p]);
        const f2 qr3 = mul2(at.q, ri3);
        ex[p] = fma2(qr3, dx, ex[p]);
        ey[p] = fma2(qr3, dy, ey[p]);
        ez[p] = fma2(qr3, dz, ez[p]);
    }
}

// PTS (cells of a z-pencil per thread, 4 or 8) is the pencil size the
// autotuner picks per system; the sums of every cell are the same for both.
template <int PTS>
__global__ void __launch_bounds__(PE_THREADS, PTS == 16 ? 3 : PTS == 8 ? 4 : 5)
k_pair_energy_grid(GridDesc g, AtomsDev a, float rho, float cfa, float rmin2,
                   float *__restrict__ U, float *__restrict__ Ex,
                   float *__restrict__ Ey, float *__restrict__ Ez)
{
    __shared__ __align__(16) AtomPairs s_at[PE_TILE];
    __shared__ float s_box[6 * (PE_THREADS / 32)];
    const int cpp = (g.nz + PTS - 1) / PTS;
    const long long t = (long long)blockIdx.x * PE_THREADS + threadIdx.x;
    const long long npen = (long long)g.nx * g.ny;
    const long long pen = t / cpp;
    const int chunk = (int)(t - pen * cpp);
    const bool live = pen < npen;
    const int i = live ? (int)(pen / g.ny) : 0;
    const int j = live ? (int)(pen - (long long)i * g.ny) : 0;
    const int k0 = chunk * PTS;
    const float px = cell_pos(i, g.cx, g.h);
    const float py = cell_pos(j, g.cy, g.h);
    float pzs[PTS];
#pragma unroll
    for (int p = 0; p < PTS; ++p) pzs[p] = cell_pos(k0 + p, g.cz, g.h);
    f2 pz[PTS / 2], lj[PTS / 2], ex[PTS / 2], ey[PTS / 2], ez[PTS / 2];
    const f2 zero = pk2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < PTS / 2; ++p) {
        pz[p] = pk2(pzs[2 * p], pzs[2 * p + 1]);
        lj[p] = ex[p] = ey[p] = ez[p] = zero;
    }
    const f2 px2 = pk2(px, px), py2 = pk2(py, py);
    // bounding box of the block's cells (padding cells included: harmless)
    float clo[3], chi[3];
    block_box(px, py, pzs[0], clo, chi, s_box);
    {
        float lo2[3], hi2[3];
        block_box(px, py, pzs[PTS - 1], lo2, hi2, s_box);
        clo[2] = fminf(clo[2], lo2[2]);
        chi[2] = fmaxf(chi[2], hi2[2]);
    }
    for (int base = 0; base < a.n; base += PE_TILE) {
        const int cnt = min(PE_TILE, a.n - base);
        __syncthreads();
        // corners of the box of the atoms this thread stages
        float tlo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, thi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
        bool have = false;
        for (int m = threadIdx.x; m < cnt; m += PE_THREADS) {
            const float4 A = a.xyzq[base + m];
            const float2 B = a.ab[base + m];
            AtomPairs at;
            at.x = pk2(A.x, A.x);
            at.y = pk2(A.y, A.y);
            at.z = pk2(A.z, A.z);
            at.q = pk2(A.w, A.w);
            at.a = pk2(B.x, B.x);
            at.nb = pk2(-B.y, -B.y);
            s_at[m] = at;
            tlo[0] = fminf(tlo[0], A.x); tlo[1] = fminf(tlo[1], A.y); tlo[2] = fminf(tlo[2], A.z);
            thi[0] = fmaxf(thi[0], A.x); thi[1] = fmaxf(thi[1], A.y); thi[2] = fmaxf(thi[2], A.z);
            have = true;
        }
        if (!have) {   // a thread without atoms repeats the tile's first one
            const float4 A = a.xyzq[base];
            tlo[0] = thi[0] = A.x; tlo[1] = thi[1] = A.y; tlo[2] = thi[2] = A.z;
        }
        // the tile needs the clamp only if the box of all its atoms comes
        // within r_min of the block's cells: the block minimum of the lower
        // corners and the block maximum of the upper corners
        float alo[3], ahi[3], unused[3];
        block_box(tlo[0], tlo[1], tlo[2], alo, unused, s_box);
        block_box(thi[0], thi[1], thi[2], unused, ahi, s_box);
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float gap = fmaxf(fmaxf(alo[c] - chi[c], clo[c] - ahi[c]), 0.f);
            d2 = fmaf(gap, gap, d2);
        }
        __syncthreads();
        if (d2 > rmin2) {
#pragma unroll 2
            for (int m = 0; m < cnt; ++m)
                energy_atom<false, PTS>(s_at[m], px2, py2, pz, rmin2, lj, ex, ey, ez);
        } else {
#pragma unroll 2
            for (int m = 0; m < cnt; ++m)
                energy_atom<true, PTS>(s_at[m], px2, py2, pz, rmin2, lj, ex, ey, ez);
        }
    }
    if (!live) return;
    const long long row = pen * g.nz;
#pragma unroll
    for (int p = 0; p < PTS / 2; ++p) {
        float l[2], x[2], y[2], z[2];
        upk2(lj[p], l[0], l[1]);
        upk2(ex[p], x[0], x[1]);
        upk2(ey[p], y[0], y[1]);
        upk2(ez[p], z[0], z[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = k0 + 2 * p + h;
            if (k < g.nz) {
                const long long idx = row + k;
                const float e2 = fmaf(x[h], x[h], fmaf(y[h], y[h], z[h] * z[h]));
                U[idx] = fmaf(cfa, e2, rho * l[h]);
                Ex[idx] = x[h];
                Ey[idx] = y[h];
                Ez[idx] = z[h];
            }
        }
    }
}

void launch_pair_energy_grid(const GridDesc &g, const AtomsDev &a, float rho,
                             float cfa, float rmin2, float *U, float *Ex,
                             float *Ey, float *Ez, int pts, cudaStream_t st)
{
    const int P = pts == 4 ? 4 : pts == 16 ? 16 : 8;
    const long long cpp = (g.nz + P - 1) / P;
    const long long threads = (long long)g.nx * g.ny * cpp;
    const long long blocks = (threads + PE_THREADS - 1) / PE_THREADS;
    count_launch();
    if (P == 4)
        k_pair_energy_grid<4><<<(unsigned)blocks, PE_THREADS, 0, st>>>(
            g, a, rho, cfa, rmin2, U, Ex, Ey, Ez);
    else if (P == 16)
        k_pair_energy_grid<16><<<(unsigned)blocks, PE_THREADS, 0, st>>>(
            g, a, rho, cfa, rmin2, U, Ex, Ey, Ez);
    else
        k_pair_energy_grid<8><<<(unsigned)blocks, PE_THREADS, 0, st>>>(
            g, a, rho, cfa, rmin2, U, Ex, Ey, Ez);
}

// ------------------------------------------------------------ block sums
// Fixed-order block reduction of a double (warp tree, then warp 0).
template <int NT>
__device__ double block_sum(double v, double *s_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s_red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (l < NT / 32) ? s_red[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;   // valid in thread 0
}

// ----------------------------------------------------- far-field nodes
constexpr int PT_THREADS = 128;

int point_energy_blocks(int np) { return (np + PT_THREADS - 1) / PT_THREADS; }

__global__ void __launch_bounds__(PT_THREADS)
k_point_energy(const float4 *__restrict__ pts, const double *__restrict__ w,
               int np, AtomsDev a, float rho, float cfa, float rmin2,
               float4 *__restrict__ UE, double *__restrict__ part)
{
    __shared__ float4 s_xyzq[PE_TILE];
    __shared__ float2 s_ab[PE_TILE];
    __shared__ double s_red[PT_THREADS / 32];
    const int k = blockIdx.x * PT_THREADS + threadIdx.x;
    const float4 P = (k < np) ? pts[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    float lj = 0.f, ex = 0.f, ey = 0.f, ez = 0.f;
    for (int base = 0; base < a.n; base += PE_TILE) {
        const int cnt = min(PE_TILE, a.n - base);
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += PT_THREADS) {
            s_xyzq[m] = a.xyzq[base + m];
            s_ab[m] = a.ab[base + m];
        }
        __syncthreads();
        for (int m = 0; m < cnt; ++m) {
            const float4 A = s_xyzq[m];
            const float2 B = s_ab[m];
            const float dx = P.x - A.x, dy = P.y - A.y, dz = P.z - A.z;
            const float r2 = fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), rmin2);
            const float ri = rsqrt_ftz(r2);
            const float ri2 = ri * ri, ri3 = ri2 * ri, ri6 = ri3 * ri3;
            lj = fmaf(ri6, fmaf(B.x, ri6, -B.y), lj);
            const float qr3 = A.w * ri3;
            ex = fmaf(qr3, dx, ex);
            ey = fmaf(qr3, dy, ey);
            ez = fmaf(qr3, dz, ez);
        }
    }
    double contrib = 0.0;
    if (k < np) {
        const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const float u = fmaf(cfa, e2, rho * lj);
        UE[k] = make_float4(ex, ey, ez, u);
        contrib = w[k] * (double)u;
    }
    const double s = block_sum<PT_THREADS>(contrib, s_red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

void launch_point_energy(const float4 *pts, const double *w, int np,
                         const AtomsDev &a, float rho, float cfa, float rmin2,
                         float4 *UE, double *part, cudaStream_t st)
{
    count_launch();
    k_point_energy<<<point_energy_blocks(np), PT_THREADS, 0, st>>>(
        pts, w, np, a, rho, cfa, rmin2, UE, part);
}

// ------------------------------------------------------ grid -> atoms
constexpr int PF_THREADS = 128;
constexpr int PF_APT = 4;                    // atoms per thread of the point kernel
constexpr int PF_ATOMS = PF_THREADS * PF_APT;
constexpr int PF_STAGE = 256;                // cells staged per pass

ForcePlan plan_pair_force(long long G, int natoms, int nsm, int apt)
{
    ForcePlan fp;
    fp.apt = apt == 2 ? 2 : 4;
    // Cell groups: a small solute fills few of a block's 512 atom slots, so
    // the block splits into cg groups of 128 / cg threads that hold the same
    // atoms and share each staged set of cells.  cg depends only on the atom
    // count (the fill of 512 / cg-atom tiles against the staging a block
    // then spreads over fewer atoms), so both atom tiles sum every atom's
    // cells in the same groups and order and stay bit-identical.
    fp.cg = 1;
    {
        double best = 0.0;
        for (int cg = 1; cg <= 4; cg *= 2) {
            const long long slots = PF_ATOMS / cg;
            const double fill = (double)natoms / (double)(slots * ((natoms + slots - 1) / slots));
            const double score = fill / (1.0 + 0.05 * cg);
            if (score > best + 1e-12) {
                best = score;
                fp.cg = cg;
            }
        }
    }
    const int per_tile = PF_THREADS / fp.cg * fp.apt;
    fp.atom_tiles = (natoms + per_tile - 1) / per_tile;
    // The cell chunks are sized from the 512-atom tile count whatever the
    // atom tile, so every atom sums the same stages in the same order and
    // both variants give bit-identical gradients.
    const long long tiles512 = (natoms + PF_ATOMS - 1) / PF_ATOMS;
    const long long target = (long long)nsm * 8 * 4;
    long long nchunk = target / tiles512;
    // Every chunk writes an FP64 partial per atom.  On small grids one-stage
    // chunks made those partials (and their reduction) cost more than the
    // pairs, so a chunk spans at least 8 stages - unless that leaves fewer
    // than two waves of blocks (counted with the 4-atom tiles, so that the
    // plan depends on the atom count alone).
    const long long tiles_ref = (natoms + PF_ATOMS / fp.cg - 1) / (PF_ATOMS / fp.cg);
    const long long fill = ((long long)nsm * 8 + tiles_ref - 1) / tiles_ref;
    const long long maxc = std::min((G + PF_STAGE - 1) / PF_STAGE,
                                    std::max(fill, G / ((long long)PF_STAGE * 8)));
    if (nchunk < 1) nchunk = 1;
    if (nchunk > maxc) nchunk = maxc;
    long long len = (G + nchunk - 1) / nchunk;
    len = (len + PF_STAGE - 1) / PF_STAGE * PF_STAGE;
    fp.chunk_len = len;
    fp.nchunk = (int)((G + len - 1) / len);
    return fp;
}

// One pair's contribution to the gradient of atom (ax, ay, az) with
// coefficients c1 = 12 rho A, c2 = -6 rho B, kq = -2 C Q, kq3 = 3 kq; E is
// the field at the point.  Without the clamp:
//   f += [r^-8 (c1 r^-6 + c2) - kq3 r^-5 (d.E)] d + kq r^-3 E.
// With it, the LJ part and the d d^T part vanish where r < r_min.
template <bool CLAMP>
__device__ __forceinline__ void force_pair(float px, float py, float pz,
                                           const float4 &E, float ax, float ay,
                                           float az, float c1, float c2,
                                           float kq, float kq3, float rmin2,
                                           float &fx, float &fy, float &fz)
{
    const float dx = px - ax, dy = py - ay, dz = pz - az;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float ri, c1m = c1, c2m = c2, k3m = kq3;
    if (CLAMP) {
        const bool un = r2 >= rmin2;                // not clamped
        ri = rsqrt_ftz(fmaxf(r2, rmin2));
        c1m = un ? c1 : 0.f;
        c2m = un ? c2 : 0.f;
        k3m = un ? kq3 : 0.f;
    } else {
        ri = rsqrt_ftz(r2);
    }
    const float ri2 = ri * ri;
    const float ri3 = ri2 * ri;
    const float ri6 = ri3 * ri3;
    const float ri8 = ri6 * ri2;
    const float glj = fmaf(c1m, ri6, c2m) * ri8;
    const float dE = fmaf(dx, E.x, fmaf(dy, E.y, dz * E.z));
    const float am = kq * ri3;
    const float cd = fmaf(-(k3m * ri3), dE * ri2, glj);
    fx = fmaf(cd, dx, fmaf(am, E.x, fx));
    fy = fmaf(cd, dy, fmaf(am, E.y, fy));
    fz = fmaf(cd, dz, fmaf(am, E.z, fz));
}

// The grid kernel's form of the same pair, for the thread's two atoms at
// once (packed pairs; nk3 = -3 kq).  The cells of one z-pencil share x and
// y, so dx, dy and dx^2 + dy^2 come in once per pencil, and the pencil's sum
// of cd d_x is dx times its sum of cd.  With r^-8 (c1 r^-6 + c2) + nk3 r^-5
// (d.E) = r^-5 [r^-3 (c1 r^-6 + c2) + nk3 (d.E)], a pair adds
//   sc += cd,  fz += cd dz,  g += r^-3 E     (the E part times kq at the end)
// in 18 packed operations.  Clamped pairs keep only r^-3 E.
struct CellQuad {
    f2 z, ex, ey, ez;   // cell z and field, each duplicated into both halves
};

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <bool CLAMP>
__device__ __forceinline__ void grad_pair2(const CellQuad &c, f2 dx, f2 dy, f2 dxy2, f2 az,
                                           f2 c1, f2 c2, f2 nk3, float rmin2, f2 &sc,
                                           f2 &fz, f2 &gx, f2 &gy, f2 &gz)
{
    const f2 dz = sub2(c.z, az);
    const f2 r2 = fma2(dz, dz, dxy2);
    float ra, rb;
    upk2(r2, ra, rb);
    f2 ri;
    bool ua = true, ub = true;   // not clamped
    if (CLAMP) {
        ua = ra >= rmin2;
        ub = rb >= rmin2;
        ri = pk2(rsqrt_ftz(fmaxf(ra, rmin2)), rsqrt_ftz(fmaxf(rb, rmin2)));
    } else {
        ri = pk2(rsqrt_ftz(ra), rsqrt_ftz(rb));
    }
    const f2 ri2 = mul2(ri, ri);
    const f2 ri3 = mul2(ri2, ri);
    const f2 ri6 = mul2(ri3, ri3);
    const f2 ri5 = mul2(ri3, ri2);
    const f2 t1 = fma2(c1, ri6, c2);
    const f2 dE = fma2(dx, c.ex, fma2(dy, c.ey, mul2(dz, c.ez)));
    f2 cd = mul2(ri5, fma2(ri3, t1, mul2(nk3, dE)));
    if (CLAMP) {
        float ca, cb;
        upk2(cd, ca, cb);
        cd = pk2(ua ? ca : 0.f, ub ? cb : 0.f);
    }
    sc = add2(sc, cd);
    fz = fma2(cd, dz, fz);
    gx = fma2(ri3, c.ex, gx);
    gy = fma2(ri3, c.ey, gy);
    gz = fma2(ri3, c.ez, gz);
}

// hi + lo += v with the rounding error of the addition kept in lo (Knuth's
// two-sum, both halves of the pairs at once)
__device__ __forceinline__ void two_sum_acc(f2 &hi, f2 &lo, f2 v)
{
    const f2 s = add2(hi, v);
    const f2 bb = sub2(s, hi);
    lo = add2(lo, add2(sub2(hi, sub2(s, bb)), sub2(v, bb)));
    hi = s;
}

// Number of solvent cells among the first n slots of a stage, from the
// stage's per-warp ballots (slot order) and their counts.
__device__ __forceinline__ int stage_rank(int n, const int *wc, const unsigned *bal)
{
    constexpr int NWORD = 2 * PF_THREADS / 32;
    const int w = n >> 5;
    int r = 0;
#pragma unroll
    for (int v = 0; v < NWORD; ++v) r += v < w ? wc[v] : 0;
    if (w < NWORD) r += __popc(bal[w] & ((1u << (n & 31)) - 1u));
    return r;
}

// APT (atoms per thread, 2 or 4, in packed pairs) is the atom tile the
// autotuner picks per system.
template <int APT, int CG>
__global__ void __launch_bounds__(PF_THREADS)
k_pair_force_grid(GridDesc g, long long G, long long chunk_len,
                  const uint8_t *__restrict__ chi, const float *__restrict__ Ex,
                  const float *__restrict__ Ey, const float *__restrict__ Ez,
                  AtomsDev a, float rmin2, double *__restrict__ part,
                  unsigned long long *__restrict__ nsolvent)
{
    static_assert(APT % 2 == 0, "a thread's atoms form packed pairs");
    constexpr int PAIRS = APT / 2;
    // CG groups of T threads: thread lt of group grp holds the tile's atoms
    // lt, lt + T, ... and visits the cells grp, grp + CG, ... of each stage
    constexpr int T = PF_THREADS / CG;
    const int grp = threadIdx.x / T, lt = threadIdx.x - grp * T;
    constexpr int ATOMS = T * APT;
    __shared__ __align__(16) CellQuad s_c[PF_STAGE];
    __shared__ int s_wc[2 * PF_THREADS / 32];
    __shared__ unsigned s_bal[2 * PF_THREADS / 32];
    __shared__ float s_box[6 * (PF_THREADS / 32)];
    // the atom tile varies fastest in launch order: the blocks of one cell
    // chunk run together and its labels and field come from DRAM once
    const int chunk = blockIdx.y;
    const int tile = blockIdx.x;
    const long long c0 = (long long)chunk * chunk_len;
    const long long c1 = min(G, c0 + chunk_len);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = PF_THREADS / 32;

    float ax[APT], ay[APT], az[APT], k1[APT], k2[APT], kq[APT],
        kq3[APT];
    int an[APT];
    const float4 A0 = a.xyzq[tile * ATOMS];   // exists: tiles are non-empty
#pragma unroll
    for (int u = 0; u < APT; ++u) {
        an[u] = tile * ATOMS + u * T + lt;
        if (an[u] < a.n) {
            const float4 A = a.xyzq[an[u]];
            const float4 F = a.fcoef[an[u]];
            ax[u] = A.x; ay[u] = A.y; az[u] = A.z;
            k1[u] = F.x; k2[u] = F.y; kq[u] = F.z;
        } else {   // idle slot: sits on a real atom and adds nothing
            ax[u] = A0.x; ay[u] = A0.y; az[u] = A0.z;
            k1[u] = k2[u] = kq[u] = 0.f;
        }
        kq3[u] = 3.f * kq[u];
    }
    // bounding box of the block's atoms
    float alo[3], ahi[3];
    block_box(ax[0], ay[0], az[0], alo, ahi, s_box);
#pragma unroll
    for (int u = 1; u < APT; ++u) {
        float lo2[3], hi2[3];
        block_box(ax[u], ay[u], az[u], lo2, hi2, s_box);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            alo[c] = fminf(alo[c], lo2[c]);
            ahi[c] = fmaxf(ahi[c], hi2[c]);
        }
    }
    f2 ax2[PAIRS], ay2[PAIRS], az2[PAIRS], c12[PAIRS], c22[PAIRS], kq2[PAIRS],
        nk32[PAIRS];
#pragma unroll
    for (int pp = 0; pp < PAIRS; ++pp) {
        const int u = 2 * pp;
        ax2[pp] = pk2(ax[u], ax[u + 1]);
        ay2[pp] = pk2(ay[u], ay[u + 1]);
        az2[pp] = pk2(az[u], az[u + 1]);
        c12[pp] = pk2(k1[u], k1[u + 1]);
        c22[pp] = pk2(k2[u], k2[u + 1]);
        kq2[pp] = pk2(kq[u], kq[u + 1]);
        nk32[pp] = pk2(-kq3[u], -kq3[u + 1]);
    }
    const f2 zero2 = pk2(0.f, 0.f);
    // the stage sums add into double-float (hi + lo) accumulators: exact
    // FP32 error-free additions instead of FP64 arithmetic, which this part
    // runs at a small fraction of the FP32 rate
    f2 shi[PAIRS][3], slo[PAIRS][3];
#pragma unroll
    for (int pp = 0; pp < PAIRS; ++pp)
#pragma unroll
        for (int c = 0; c < 3; ++c) shi[pp][c] = slo[pp][c] = zero2;

    const long long nyz = (long long)g.ny * g.nz;
    unsigned long long seen = 0;
    for (long long s = c0; s < c1; s += PF_STAGE) {
        // stage the solvent cells of [s, s + PF_STAGE) in index order
        bool v[2];
        float4 P[2], Ev[2];
#pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
            long long idx = s + hlf * PF_THREADS + threadIdx.x;
            v[hlf] = (idx < c1) && chi[idx] == 0;
            if (idx >= c1) idx = s;          // position only feeds the box
            const int i = (int)(idx / nyz);
            const long long rem = idx - (long long)i * nyz;
            const int j = (int)(rem / g.nz);
            const int k = (int)(rem - (long long)j * g.nz);
            P[hlf] = make_float4(cell_pos(i, g.cx, g.h), cell_pos(j, g.cy, g.h),
                                 cell_pos(k, g.cz, g.h), 0.f);
            if (v[hlf]) Ev[hlf] = make_float4(Ex[idx], Ey[idx], Ez[idx], 0.f);
        }
        // the stage needs the clamp only if its cells' box comes within r_min
        // of the block's atoms
        float clo[3], chi3[3], lo2[3], hi2[3];
        block_box(P[0].x, P[0].y, P[0].z, clo, chi3, s_box);
        block_box(P[1].x, P[1].y, P[1].z, lo2, hi2, s_box);
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float lo = fminf(clo[c], lo2[c]), hi = fmaxf(chi3[c], hi2[c]);
            const float gap = fmaxf(fmaxf(alo[c] - hi, lo - ahi[c]), 0.f);
            d2 = fmaf(gap, gap, d2);
        }
        const bool clamp = !(d2 > rmin2);
        const unsigned b0 = __ballot_sync(0xffffffffu, v[0]);
        const unsigned b1 = __ballot_sync(0xffffffffu, v[1]);
        __syncthreads();   // previous pass finished reading s_p / s_e
        if (lane == 0) {
            s_wc[warp] = __popc(b0);
            s_wc[NW + warp] = __popc(b1);
            s_bal[warp] = b0;
            s_bal[NW + warp] = b1;
        }
        __syncthreads();
        int off0 = 0, off1 = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < 2 * NW; ++w) {
            const int c = s_wc[w];
            if (w < warp) off0 += c;
            if (w < NW + warp) off1 += c;
            tot += c;
        }
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
            if (!v[hlf]) continue;
            const int pos = (hlf ? off1 + __popc(b1 & lt) : off0 + __popc(b0 & lt));
            CellQuad cp;
            cp.z = pk2(P[hlf].z, P[hlf].z);
            cp.ex = pk2(Ev[hlf].x, Ev[hlf].x);
            cp.ey = pk2(Ev[hlf].y, Ev[hlf].y);
            cp.ez = pk2(Ev[hlf].z, Ev[hlf].z);
            s_c[pos] = cp;
        }
        __syncthreads();
        seen += (unsigned long long)tot;
        f2 fx[PAIRS], fy[PAIRS], fz[PAIRS], gx[PAIRS], gy[PAIRS], gz[PAIRS];
#pragma unroll
        for (int pp = 0; pp < PAIRS; ++pp) fx[pp] = fy[pp] = fz[pp] = gx[pp] = gy[pp] = gz[pp] = zero2;
        // the stage's cells by z-pencil: the solvent cells of pencil pen sit
        // at positions [st, en) of the compacted list
        const long long lim = min((long long)PF_STAGE, c1 - s);
        const long long pen_end = (s + lim - 1) / g.nz;
        for (long long pen = s / g.nz; pen <= pen_end; ++pen) {
            const int st = stage_rank((int)max(pen * g.nz - s, 0LL), s_wc, s_bal);
            const int en = stage_rank((int)min((pen + 1) * g.nz - s, lim), s_wc, s_bal);
            if (st == en) continue;
            const int i = (int)(pen / g.ny);
            const int j = (int)(pen - (long long)i * g.ny);
            const float x = cell_pos(i, g.cx, g.h), y = cell_pos(j, g.cy, g.h);
            const f2 x2 = pk2(x, x), y2 = pk2(y, y);
            f2 dx[PAIRS], dy[PAIRS], dxy2[PAIRS], sc[PAIRS];
#pragma unroll
            for (int pp = 0; pp < PAIRS; ++pp) {
                dx[pp] = sub2(x2, ax2[pp]);
                dy[pp] = sub2(y2, ay2[pp]);
                dxy2[pp] = fma2(dx[pp], dx[pp], mul2(dy[pp], dy[pp]));
                sc[pp] = zero2;
            }
            const int first = st + ((grp - st) & (CG - 1));
            if (clamp) {
#pragma unroll 4
                for (int p = first; p < en; p += CG) {
                    const CellQuad c = s_c[p];
#pragma unroll
                    for (int pp = 0; pp < PAIRS; ++pp)
                        grad_pair2<true>(c, dx[pp], dy[pp], dxy2[pp], az2[pp], c12[pp], c22[pp],
                                         nk32[pp], rmin2, sc[pp], fz[pp], gx[pp], gy[pp], gz[pp]);
                }
            } else {
#pragma unroll 4
                for (int p = first; p < en; p += CG) {
                    const CellQuad c = s_c[p];
#pragma unroll
                    for (int pp = 0; pp < PAIRS; ++pp)
                        grad_pair2<false>(c, dx[pp], dy[pp], dxy2[pp], az2[pp], c12[pp], c22[pp],
                                          nk32[pp], rmin2, sc[pp], fz[pp], gx[pp], gy[pp], gz[pp]);
                }
            }
#pragma unroll
            for (int pp = 0; pp < PAIRS; ++pp) {
                fx[pp] = fma2(sc[pp], dx[pp], fx[pp]);
                fy[pp] = fma2(sc[pp], dy[pp], fy[pp]);
            }
        }
#pragma unroll
        for (int pp = 0; pp < PAIRS; ++pp) {
            two_sum_acc(shi[pp][0], slo[pp][0], fma2(kq2[pp], gx[pp], fx[pp]));
            two_sum_acc(shi[pp][1], slo[pp][1], fma2(kq2[pp], gy[pp], fy[pp]));
            two_sum_acc(shi[pp][2], slo[pp][2], fma2(kq2[pp], gz[pp], fz[pp]));
        }
    }
    double acc[APT][3];
#pragma unroll
    for (int pp = 0; pp < PAIRS; ++pp)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float h0, h1, l0, l1;
            upk2(shi[pp][c], h0, h1);
            upk2(slo[pp][c], l0, l1);
            acc[2 * pp][c] = (double)h0 + (double)l0;
            acc[2 * pp + 1][c] = (double)h1 + (double)l1;
        }
    if (CG > 1) {     // the groups' sums, added in group order
        __shared__ double s_acc[PF_THREADS * 4 * 3];
#pragma unroll
        for (int u = 0; u < APT; ++u)
#pragma unroll
            for (int c = 0; c < 3; ++c) s_acc[(threadIdx.x * APT + u) * 3 + c] = acc[u][c];
        __syncthreads();
        if (grp == 0) {
#pragma unroll
            for (int u = 0; u < APT; ++u)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double t = 0.0;
                    for (int q = 0; q < CG; ++q) t += s_acc[((q * T + lt) * APT + u) * 3 + c];
                    acc[u][c] = t;
                }
        }
    }
    if (grp == 0) {
#pragma unroll
        for (int u = 0; u < APT; ++u) {
            if (an[u] < a.n) {
                double *o = part + ((long long)chunk * a.n + an[u]) * 3;
                o[0] = acc[u][0];
                o[1] = acc[u][1];
                o[2] = acc[u][2];
            }
        }
    }
    if (nsolvent && tile == 0 && threadIdx.x == 0) atomicAdd(nsolvent, seen);
}

void launch_pair_force_grid(const GridDesc &g, const ForcePlan &fp,
                            const uint8_t *chi, const float *Ex,
                            const float *Ey, const float *Ez,
                            const AtomsDev &a, float rmin2, double *part,
                            unsigned long long *nsolvent, cudaStream_t st)
{
    const long long G = (long long)g.nx * g.ny * g.nz;
    dim3 grid(fp.atom_tiles, fp.nchunk);
    count_launch();
#define VESIS_FORCE_LAUNCH(A, C)                                                            \
    k_pair_force_grid<A, C><<<grid, PF_THREADS, 0, st>>>(g, G, fp.chunk_len, chi, Ex, Ey, Ez, a, \
                                                         rmin2, part, nsolvent)
    if (fp.apt == 2) {
        if (fp.cg == 4) VESIS_FORCE_LAUNCH(2, 4);
        else if (fp.cg == 2) VESIS_FORCE_LAUNCH(2, 2);
        else VESIS_FORCE_LAUNCH(2, 1);
    } else {
        if (fp.cg == 4) VESIS_FORCE_LAUNCH(4, 4);
        else if (fp.cg == 2) VESIS_FORCE_LAUNCH(4, 2);
        else VESIS_FORCE_LAUNCH(4, 1);
    }
#undef VESIS_FORCE_LAUNCH
}

// Far-field nodes -> atoms: weighted points, all of them solvent.
ForcePlan plan_point_force(int np, int natoms, int nsm)
{
    ForcePlan fp;
    fp.apt = PF_APT;
    fp.cg = 1;
    fp.atom_tiles = (natoms + PF_ATOMS - 1) / PF_ATOMS;
    long long nchunk = ((long long)nsm * 8) / fp.atom_tiles;
    const long long maxc = (np + PF_STAGE - 1) / PF_STAGE;
    if (nchunk < 1) nchunk = 1;
    if (nchunk > maxc) nchunk = maxc;
    long long len = (np + nchunk - 1) / nchunk;
    len = (len + PF_STAGE - 1) / PF_STAGE * PF_STAGE;
    fp.chunk_len = len;
    fp.nchunk = (int)((np + len - 1) / len);
    return fp;
}

__global__ void __launch_bounds__(PF_THREADS)
k_point_force(const float4 *__restrict__ pts, const float *__restrict__ wf,
              int np, const float4 *__restrict__ UE, long long chunk_len,
              AtomsDev a, float rmin2, double *__restrict__ part)
{
    __shared__ float4 s_p[PF_STAGE];
    __shared__ float4 s_e[PF_STAGE];
    const int chunk = blockIdx.y;   // atom tiles fastest, as in k_pair_force_grid
    const int tile = blockIdx.x;
    const long long c0 = (long long)chunk * chunk_len;
    const long long c1 = min((long long)np, c0 + chunk_len);
    float ax[PF_APT], ay[PF_APT], az[PF_APT], k1[PF_APT], k2[PF_APT], kq[PF_APT];
    int an[PF_APT];
#pragma unroll
    for (int u = 0; u < PF_APT; ++u) {
        an[u] = tile * PF_ATOMS + u * PF_THREADS + threadIdx.x;
        if (an[u] < a.n) {
            const float4 A = a.xyzq[an[u]];
            const float4 F = a.fcoef[an[u]];
            ax[u] = A.x; ay[u] = A.y; az[u] = A.z;
            k1[u] = F.x; k2[u] = F.y; kq[u] = F.z;
        } else {
            ax[u] = ay[u] = az[u] = 0.f;
            k1[u] = k2[u] = kq[u] = 0.f;
        }
    }
    double acc[PF_APT][3];
#pragma unroll
    for (int u = 0; u < PF_APT; ++u) acc[u][0] = acc[u][1] = acc[u][2] = 0.0;
    for (long long s = c0; s < c1; s += PF_STAGE) {
        const int cnt = (int)min((long long)PF_STAGE, c1 - s);
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += PF_THREADS) {
            float4 P = pts[s + m];
            P.w = wf[s + m];
            s_p[m] = P;
            s_e[m] = UE[s + m];
        }
        __syncthreads();
        float f[PF_APT][3];
#pragma unroll
        for (int u = 0; u < PF_APT; ++u) f[u][0] = f[u][1] = f[u][2] = 0.f;
        for (int p = 0; p < cnt; ++p) {
            const float4 Pp = s_p[p];
            const float4 Ep = s_e[p];
#pragma unroll
            for (int u = 0; u < PF_APT; ++u) {
                float gx = 0.f, gy = 0.f, gz = 0.f;
                force_pair<true>(Pp.x, Pp.y, Pp.z, Ep, ax[u], ay[u], az[u], k1[u],
                                 k2[u], kq[u], 3.f * kq[u], rmin2, gx, gy, gz);
                f[u][0] = fmaf(Pp.w, gx, f[u][0]);
                f[u][1] = fmaf(Pp.w, gy, f[u][1]);
                f[u][2] = fmaf(Pp.w, gz, f[u][2]);
            }
        }
#pragma unroll
        for (int u = 0; u < PF_APT; ++u) {
            acc[u][0] += (double)f[u][0];
            acc[u][1] += (double)f[u][1];
            acc[u][2] += (double)f[u][2];
        }
    }
#pragma unroll
    for (int u = 0; u < PF_APT; ++u) {
        if (an[u] < a.n) {
            double *o = part + ((long long)chunk * a.n + an[u]) * 3;
            o[0] = acc[u][0];
            o[1] = acc[u][1];
            o[2] = acc[u][2];
        }
    }
}

void launch_point_force(const float4 *pts, const float *wf, int np,
                        const float4 *UE, const ForcePlan &fp,
                        const AtomsDev &a, float rmin2, double *part,
                        cudaStream_t st)
{
    dim3 grid(fp.atom_tiles, fp.nchunk);
    count_launch();
    k_point_force<<<grid, PF_THREADS, 0, st>>>(pts, wf, np, UE, fp.chunk_len,
                                               a, rmin2, part);
}

// ------------------------------------------------------ ordered reductions
__global__ void k_force_reduce(const double *__restrict__ part, int nchunk,
                               int natoms, double scale, double *__restrict__ out,
                               int accumulate)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n3 = natoms * 3;
    if (t >= n3) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)c * n3 + t];
    s *= scale;
    out[t] = accumulate ? out[t] + s : s;
}

void launch_force_reduce(const double *part, int nchunk, int natoms,
                         double scale, double *out, int accumulate,
                         cudaStream_t st)
{
    const int n3 = natoms * 3;
    count_launch();
    k_force_reduce<<<(n3 + 255) / 256, 256, 0, st>>>(part, nchunk, natoms,
                                                     scale, out, accumulate);
}

__global__ void __launch_bounds__(1024)
k_sum_doubles(const double *__restrict__ in, int n, double *out, int accumulate)
{
    __shared__ double s_red[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 1024) v += in[i];
    const double s = block_sum<1024>(v, s_red);
    if (threadIdx.x == 0) out[0] = accumulate ? out[0] + s : s;
}

void launch_sum_doubles(const double *in, int n, double *out, int accumulate,
                        cudaStream_t st)
{
    count_launch();
    k_sum_doubles<<<1, 1024, 0, st>>>(in, n, out, accumulate);
}

}  // namespace vesis
