// Binary level-set sweep kernels (Sec. 3.1, Step 2) for sm_103a.
//
// Surface energy with the separable Gaussian kernel g(a,b,c) = q_a q_b q_c /
// 256^3 (q integer, sum 256): E_s = c sum_j chi_j (1 - w_j), w = g * chi with
// cells outside the box counted as solvent.  W = 256^3 w is computed in
// three integer passes (z, y, x), so it is exact: pass 1 <= 256, pass 2
// <= 2^16, pass 3 <= 2^24.
//
// This file holds the full-grid passes (convolution, flip energies, energy
// sums, initial labels); the flip rounds themselves run in sweep.cu.
#include "vesis_internal.cuh"

namespace vesis {

constexpr int CT = 256;   // threads per block of the cell-parallel kernels

// y and x passes: 1 = shared-memory tiles, 0 = register walks
#ifndef VESIS_CONV_TILE
#define VESIS_CONV_TILE 1
#endif

static unsigned cell_blocks(const GridDesc &g)
{
    const long long G = (long long)g.nx * g.ny * g.nz;
    return (unsigned)((G + CT - 1) / CT);
}

// The 1-D weights centred in 17 entries (q17[8 + a] = q_a, zero for
// |a| > r), so every pass runs the same 17-tap loop for any r <= 8.
struct Q17 {
    int q[2 * kMaxR + 1];
};

static Q17 centred(const KernelW &kw)
{
    Q17 w{};
    for (int a = -kw.r; a <= kw.r; ++a) w.q[kMaxR + a] = kw.q[a + kw.r];
    return w;
}

// z pass, any layout: one thread per cell.
__global__ void k_conv_z(GridDesc g, Q17 w, const uint8_t *__restrict__ chi,
                         uint16_t *__restrict__ T1)
{
    const long long G = (long long)g.nx * g.ny * g.nz;
    const long long p = (long long)blockIdx.x * CT + threadIdx.x;
    if (p >= G) return;
    const int k = (int)(p % g.nz);
    unsigned s = 0;
#pragma unroll
    for (int a = -kMaxR; a <= kMaxR; ++a) {
        const int kk = k + a;
        if (kk >= 0 && kk < g.nz) s += (unsigned)w.q[a + kMaxR] * chi[p + a];
    }
    T1[p] = (uint16_t)s;
}

// z pass on rows of whole 8-cell chunks (nz % 8 == 0, chi 8-byte and T1
// 16-byte aligned): one thread per chunk reads the chunk and its two
// neighbours as three 8-byte words and writes 8 sums as one 16-byte store.
__global__ void __launch_bounds__(CT)
k_conv_z8(Q17 w, const uint8_t *__restrict__ chi, uint16_t *__restrict__ T1, int nz,
          unsigned nchunk)
{
    const unsigned t = blockIdx.x * CT + threadIdx.x;
    if (t >= nchunk) return;
    const unsigned cpr = (unsigned)nz / 8u;
    const unsigned row = t / cpr;
    const int k0 = (int)(t - row * cpr) * 8;
    const uint8_t *rp = chi + (long long)row * nz;
    const unsigned long long lo =
        k0 >= 8 ? __ldg(reinterpret_cast<const unsigned long long *>(rp + k0 - 8)) : 0ull;
    const unsigned long long mid = __ldg(reinterpret_cast<const unsigned long long *>(rp + k0));
    const unsigned long long hi =
        k0 + 8 < nz ? __ldg(reinterpret_cast<const unsigned long long *>(rp + k0 + 8)) : 0ull;
    unsigned b[24];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        b[i] = (unsigned)(lo >> (8 * i)) & 0xffu;
        b[8 + i] = (unsigned)(mid >> (8 * i)) & 0xffu;
        b[16 + i] = (unsigned)(hi >> (8 * i)) & 0xffu;
    }
    unsigned o[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {     // cell k0 + c: bytes c .. c + 16 are cells k0 + c - 8 .. + 8
        unsigned s = 0;
#pragma unroll
        for (int m = 0; m <= 2 * kMaxR; ++m) s += (unsigned)w.q[m] * b[c + m];
        o[c] = s;
    }
    *reinterpret_cast<uint4 *>(T1 + (long long)row * nz + k0) =
        make_uint4(o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16),
                   o[6] | (o[7] << 16));
}

// The z pass with byte dot products: the 17 weights, re-packed for each of
// the 8 byte alignments c of an output inside its chunk, so that output c
// is the sum over the six 4-byte words j of the chunk's 24-byte window of
// dp4a(word j, qp[c][j]) (all weights must fit in a byte).
struct QPack {
    unsigned qp[8][6];
};

static bool pack_dp4a(const Q17 &w, QPack *out)
{
    for (int m = 0; m <= 2 * kMaxR; ++m)
        if (w.q[m] < 0 || w.q[m] > 255) return false;
    for (int c = 0; c < 8; ++c)
        for (int j = 0; j < 6; ++j) {
            unsigned v = 0;
            for (int t = 0; t < 4; ++t) {
                const int m = 4 * j + t - c;     // window byte 4j + t holds tap m
                if (m >= 0 && m <= 2 * kMaxR) v |= (unsigned)w.q[m] << (8 * t);
            }
            out->qp[c][j] = v;
        }
    return true;
}

__global__ void __launch_bounds__(CT)
k_conv_z8_dp4a(QPack w, const uint8_t *__restrict__ chi, uint16_t *__restrict__ T1, int nz,
               unsigned nchunk)
{
    const unsigned t = blockIdx.x * CT + threadIdx.x;
    if (t >= nchunk) return;
    const unsigned cpr = (unsigned)nz / 8u;
    const unsigned row = t / cpr;
    const int k0 = (int)(t - row * cpr) * 8;
    const uint8_t *rp = chi + (long long)row * nz;
    const uint2 lo = k0 >= 8 ? __ldg(reinterpret_cast<const uint2 *>(rp + k0 - 8)) : make_uint2(0u, 0u);
    const uint2 mid = __ldg(reinterpret_cast<const uint2 *>(rp + k0));
    const uint2 hi = k0 + 8 < nz ? __ldg(reinterpret_cast<const uint2 *>(rp + k0 + 8))
                                 : make_uint2(0u, 0u);
    const unsigned wd[6] = {lo.x, lo.y, mid.x, mid.y, hi.x, hi.y};
    unsigned o[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        unsigned s = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (w.qp[c][j] != 0u) s = __dp4a(wd[j], w.qp[c][j], s);
        o[c] = s;
    }
    *reinterpret_cast<uint4 *>(T1 + (long long)row * nz + k0) =
        make_uint4(o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16),
                   o[6] | (o[7] << 16));
}

// y and x passes: every line along the pass axis (axis stride `as`) is
// walked by threads that each own KW adjacent z cells of it and a chunk of
// 32 outputs; 17 inputs sit in a register ring, so each input is loaded once
// per chunk and the loads of a warp are contiguous along z.  Lines: outer
// index o (stride os) x z index k; the element at axis position t is
// o * os + t * as + k.
template <typename TI>
__device__ __forceinline__ void ld_kw(const TI *p, unsigned (&v)[1])
{
    v[0] = (unsigned)__ldg(p);
}
__device__ __forceinline__ void ld_kw(const uint16_t *p, unsigned (&v)[2])
{
    const unsigned x = __ldg(reinterpret_cast<const unsigned *>(p));
    v[0] = x & 0xffffu;
    v[1] = x >> 16;
}
__device__ __forceinline__ void ld_kw(const uint32_t *p, unsigned (&v)[2])
{
    const uint2 x = __ldg(reinterpret_cast<const uint2 *>(p));
    v[0] = x.x;
    v[1] = x.y;
}
__device__ __forceinline__ void st_kw(uint32_t *p, const unsigned (&v)[1]) { *p = v[0]; }
__device__ __forceinline__ void st_kw(uint32_t *p, const unsigned (&v)[2])
{
    *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
}

constexpr int WALK = 32;   // outputs per thread along the pass axis

template <int KW, typename TI>
__global__ void __launch_bounds__(CT)
k_conv_walk(Q17 w, const TI *__restrict__ in, uint32_t *__restrict__ out, int n_axis,
            long long as, long long os, int nz, unsigned nthreads, unsigned nchunk)
{
    const unsigned t = blockIdx.x * CT + threadIdx.x;
    if (t >= nthreads) return;
    const unsigned nkq = (unsigned)nz / KW;
    const unsigned kq = t % nkq;
    const unsigned rest = t / nkq;
    const unsigned c = rest % nchunk;
    const unsigned o = rest / nchunk;
    const long long base = (long long)o * os + (long long)(kq * KW);
    const int t0 = (int)c * WALK;
    unsigned ring[2 * kMaxR + 1][KW];
#pragma unroll
    for (int s = 0; s < WALK + 2 * kMaxR; ++s) {
        const int ta = t0 - kMaxR + s;
        unsigned v[KW];
        if (ta >= 0 && ta < n_axis) {
            ld_kw(in + base + (long long)ta * as, v);
        } else {
#pragma unroll
            for (int e = 0; e < KW; ++e) v[e] = 0u;
        }
#pragma unroll
        for (int e = 0; e < KW; ++e) ring[s % (2 * kMaxR + 1)][e] = v[e];
        if (s >= 2 * kMaxR) {
            const int to = t0 + s - 2 * kMaxR;
            if (to < n_axis) {
                unsigned acc[KW];
#pragma unroll
                for (int e = 0; e < KW; ++e) acc[e] = 0u;
#pragma unroll
                for (int m = 0; m <= 2 * kMaxR; ++m)
#pragma unroll
                    for (int e = 0; e < KW; ++e)
                        acc[e] += (unsigned)w.q[m] * ring[(s - 2 * kMaxR + m) % (2 * kMaxR + 1)][e];
                st_kw(out + base + (long long)to * as, acc);
            }
        }
    }
}

// y and x passes through shared memory: a block takes 64 z cells of one
// line bundle and 64 outputs along the pass axis; its 256 threads load the
// 80 x 64 input tile (16 halo rows) with all loads in flight, then each
// thread forms 16 outputs of one z column from a 17-entry register ring.
constexpr int TK = 64, TA = 64, TR = TA + 2 * kMaxR;

template <typename TI>
__global__ void __launch_bounds__(CT)
k_conv_tile(Q17 w, const TI *__restrict__ in, uint32_t *__restrict__ out, int n_axis,
            long long as, long long os, int nz)
{
    __shared__ TI tile[TR][TK];
    const int k0 = blockIdx.x * TK, a0 = blockIdx.y * TA;
    const long long base = (long long)blockIdx.z * os;
    constexpr int PER = TR * TK / CT;            // 20 loads per thread
    TI v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * CT;
        const int row = e / TK, k = k0 + e % TK;
        const int ta = a0 - kMaxR + row;
        v[u] = (ta >= 0 && ta < n_axis && k < nz) ? __ldg(in + base + (long long)ta * as + k)
                                                  : (TI)0;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * CT;
        tile[e / TK][e % TK] = v[u];
    }
    __syncthreads();
    const int kk = threadIdx.x % TK, seg = threadIdx.x / TK;   // 4 segments of 16 outputs
    const int k = k0 + kk;
    if (k >= nz) return;
    unsigned ring[2 * kMaxR + 1];
#pragma unroll
    for (int s = 0; s < 16 + 2 * kMaxR; ++s) {
        ring[s % (2 * kMaxR + 1)] = (unsigned)tile[seg * 16 + s][kk];
        if (s >= 2 * kMaxR) {
            const int ta = a0 + seg * 16 + s - 2 * kMaxR;
            if (ta < n_axis) {
                unsigned acc = 0u;
#pragma unroll
                for (int m = 0; m <= 2 * kMaxR; ++m)
                    acc += (unsigned)w.q[m] * ring[(s - 2 * kMaxR + m) % (2 * kMaxR + 1)];
                out[base + (long long)ta * as + k] = acc;
            }
        }
    }
}

template <typename TI>
static void launch_tile(const Q17 &w, const TI *in, uint32_t *out, int n_axis, long long as,
                        long long os, int n_outer, int nz, cudaStream_t st)
{
    count_launch();
    const dim3 grid((unsigned)((nz + TK - 1) / TK), (unsigned)((n_axis + TA - 1) / TA),
                    (unsigned)n_outer);
    k_conv_tile<TI><<<grid, CT, 0, st>>>(w, in, out, n_axis, as, os, nz);
}

template <int KW, typename TI>
static void launch_walk(const Q17 &w, const TI *in, uint32_t *out, int n_axis, long long as,
                        long long os, int n_outer, int nz, cudaStream_t st)
{
    const unsigned nchunk = (unsigned)((n_axis + WALK - 1) / WALK);
    const unsigned nthreads = (unsigned)n_outer * nchunk * (unsigned)(nz / KW);
    count_launch();
    k_conv_walk<KW, TI><<<(nthreads + CT - 1) / CT, CT, 0, st>>>(w, in, out, n_axis, as, os, nz,
                                                                  nthreads, nchunk);
}

// Full 3-D stencil (the sin^2 kernel): the (2R+1)^3 weights sit in shared
// memory.  Rows of whole 8-cell chunks (nz % 8 == 0, aligned): a thread
// forms 8 sums along z; for each (a, b) row offset it loads the chunk and
// its two neighbours as three 8-byte words and applies that row's 2R+1
// weights (rows of all-zero weights are skipped, as are zero weights).
constexpr int K3MAX = (2 * kMaxR + 1) * (2 * kMaxR + 1) * (2 * kMaxR + 1);

__global__ void __launch_bounds__(CT)
k_conv3_z8(int nx, int ny, int nz, int R, const int *__restrict__ k3,
           const uint8_t *__restrict__ chi, uint32_t *__restrict__ W, unsigned nchunk)
{
    __shared__ int sk[K3MAX];
    const int w = 2 * R + 1;
    for (int e = threadIdx.x; e < w * w * w; e += CT) sk[e] = k3[e];
    __syncthreads();
    const unsigned t = blockIdx.x * CT + threadIdx.x;
    if (t >= nchunk) return;
    const unsigned cpr = (unsigned)nz / 8u;
    const unsigned row = t / cpr;
    const int k0 = (int)(t - row * cpr) * 8;
    const int i = (int)(row / (unsigned)ny), j = (int)(row - (unsigned)i * (unsigned)ny);
    unsigned acc[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (int a = -R; a <= R; ++a) {
        const int ii = i + a;
        if (ii < 0 || ii >= nx) continue;
        for (int b = -R; b <= R; ++b) {
            const int jj = j + b;
            if (jj < 0 || jj >= ny) continue;
            const int *wr = sk + ((a + R) * w + (b + R)) * w + R;   // wr[c], c = -R..R
            bool any = false;
            for (int c = -R; c <= R; ++c) any |= wr[c] != 0;
            if (!any) continue;
            const uint8_t *rp = chi + ((long long)ii * ny + jj) * nz;
            const unsigned long long lo =
                k0 >= 8 ? __ldg(reinterpret_cast<const unsigned long long *>(rp + k0 - 8)) : 0ull;
            const unsigned long long mid =
                __ldg(reinterpret_cast<const unsigned long long *>(rp + k0));
            const unsigned long long hi =
                k0 + 8 < nz ? __ldg(reinterpret_cast<const unsigned long long *>(rp + k0 + 8))
                            : 0ull;
            unsigned by[24];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                by[e] = (unsigned)(lo >> (8 * e)) & 0xffu;
                by[8 + e] = (unsigned)(mid >> (8 * e)) & 0xffu;
                by[16 + e] = (unsigned)(hi >> (8 * e)) & 0xffu;
            }
#pragma unroll
            for (int m = 0; m <= 2 * kMaxR; ++m) {     // tap c = m - 8
                const int c = m - kMaxR;
                if (c < -R || c > R) continue;
                const unsigned wt = (unsigned)wr[c];
                if (wt == 0u) continue;
#pragma unroll
                for (int o = 0; o < 8; ++o) acc[o] += wt * by[o + m];   // cell k0 + o + c
            }
        }
    }
    uint32_t *dst = W + (long long)row * nz + k0;
    reinterpret_cast<uint4 *>(dst)[0] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
    reinterpret_cast<uint4 *>(dst)[1] = make_uint4(acc[4], acc[5], acc[6], acc[7]);
}

// Any layout: one thread per cell.
__global__ void __launch_bounds__(CT)
k_conv3(GridDesc g, int R, const int *__restrict__ k3, const uint8_t *__restrict__ chi,
        uint32_t *__restrict__ W)
{
    __shared__ int sk[K3MAX];
    const int w = 2 * R + 1;
    for (int e = threadIdx.x; e < w * w * w; e += CT) sk[e] = k3[e];
    __syncthreads();
    const long long nyz = (long long)g.ny * g.nz;
    const long long G = nyz * g.nx;
    const long long p = (long long)blockIdx.x * CT + threadIdx.x;
    if (p >= G) return;
    const int i = (int)(p / nyz);
    const long long rem = p - (long long)i * nyz;
    const int j = (int)(rem / g.nz);
    const int k = (int)(rem - (long long)j * g.nz);
    unsigned s = 0u;
    for (int a = -R; a <= R; ++a) {
        if (i + a < 0 || i + a >= g.nx) continue;
        for (int b = -R; b <= R; ++b) {
            if (j + b < 0 || j + b >= g.ny) continue;
            const int *wr = sk + ((a + R) * w + (b + R)) * w + R;
            const uint8_t *rp = chi + ((long long)(i + a) * g.ny + (j + b)) * g.nz;
            for (int c = -R; c <= R; ++c) {
                if (k + c < 0 || k + c >= g.nz || wr[c] == 0) continue;
                s += (unsigned)wr[c] * rp[k + c];
            }
        }
    }
    W[p] = s;
}

__global__ void k_flip_energy(GridDesc g, const uint32_t *__restrict__ W,
                              const uint8_t *__restrict__ chi,
                              const float *__restrict__ U, FlipConst fc,
                              double *__restrict__ dE, uint8_t *__restrict__ cand)
{
    const long long nyz = (long long)g.ny * g.nz;
    const long long G = nyz * g.nx;
    const long long p = (long long)blockIdx.x * CT + threadIdx.x;
    if (p >= G) return;
    const int i = (int)(p / nyz);
    const long long rem = p - (long long)i * nyz;
    const int j = (int)(rem / g.nz);
    const int k = (int)(rem - (long long)j * g.nz);
    const bool c = is_candidate(g, chi, p, i, j, k, nyz);
    cand[p] = c;
    dE[p] = c ? flip_dE(chi[p], W[p], U[p], fc) : 0.0;
}

// ----------------------------------------------------------------- sums
int terms_blocks(long long G)
{
    long long nb = (G + CT - 1) / CT;
    return (int)(nb < 1024 ? nb : 1024);
}

__global__ void __launch_bounds__(CT)
k_terms(GridDesc g, const uint8_t *__restrict__ chi, const uint32_t *__restrict__ W,
        const float *__restrict__ U, const float *__restrict__ Ex,
        const float *__restrict__ Ey, const float *__restrict__ Ez, float cfa,
        unsigned ksum, long long *__restrict__ part_s, double *__restrict__ part_v,
        double *__restrict__ part_c)
{
    __shared__ long long s_s[CT / 32], s_n[CT / 32];
    __shared__ double s_v[CT / 32], s_c[CT / 32];
    const long long G = (long long)g.nx * g.ny * g.nz;
    long long S = 0, N = 0;
    double V = 0.0, Cs = 0.0;
    const long long stride = (long long)gridDim.x * CT;
    for (long long p = (long long)blockIdx.x * CT + threadIdx.x; p < G; p += stride) {
        if (chi[p]) {
            S += (long long)ksum - (long long)W[p];
            N += 1;
        } else {
            V += (double)U[p];
            if (Ex) {
                const float ex = Ex[p], ey = Ey[p], ez = Ez[p];
                Cs += (double)(cfa * fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S += __shfl_down_sync(0xffffffffu, S, o);
        N += __shfl_down_sync(0xffffffffu, N, o);
        V += __shfl_down_sync(0xffffffffu, V, o);
        Cs += __shfl_down_sync(0xffffffffu, Cs, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_s[w] = S;
        s_n[w] = N;
        s_v[w] = V;
        s_c[w] = Cs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ts = 0, tn = 0;
        double tv = 0.0, tc = 0.0;
        for (int q = 0; q < CT / 32; ++q) {
            ts += s_s[q];
            tn += s_n[q];
            tv += s_v[q];
            tc += s_c[q];
        }
        part_s[2 * blockIdx.x] = ts;
        part_s[2 * blockIdx.x + 1] = tn;
        part_v[blockIdx.x] = tv;
        part_c[blockIdx.x] = tc;
    }
}

// One block of 1024 threads, nb <= 1024 partials: integer sums are exact;
// the FP64 sums follow a fixed tree (warp shuffles, then warp 0), so the
// result does not depend on timing.
__global__ void __launch_bounds__(1024)
k_terms_final(const long long *__restrict__ part_s, const double *__restrict__ part_v,
              const double *__restrict__ part_c, int nb, double c, double D3,
              double h3, double *out)
{
    __shared__ long long s_S[32], s_N[32];
    __shared__ double s_V[32], s_C[32];
    const int b = threadIdx.x, lane = b & 31, w = b >> 5;
    long long S = 0, N = 0;
    double V = 0.0, Cs = 0.0;
    if (b < nb) {
        S = part_s[2 * b];
        N = part_s[2 * b + 1];
        V = part_v[b];
        Cs = part_c[b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S += __shfl_down_sync(0xffffffffu, S, o);
        N += __shfl_down_sync(0xffffffffu, N, o);
        V += __shfl_down_sync(0xffffffffu, V, o);
        Cs += __shfl_down_sync(0xffffffffu, Cs, o);
    }
    if (lane == 0) {
        s_S[w] = S;
        s_N[w] = N;
        s_V[w] = V;
        s_C[w] = Cs;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        S = lane < nw ? s_S[lane] : 0;
        N = lane < nw ? s_N[lane] : 0;
        V = lane < nw ? s_V[lane] : 0.0;
        Cs = lane < nw ? s_C[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            S += __shfl_down_sync(0xffffffffu, S, o);
            N += __shfl_down_sync(0xffffffffu, N, o);
            V += __shfl_down_sync(0xffffffffu, V, o);
            Cs += __shfl_down_sync(0xffffffffu, Cs, o);
        }
        if (lane == 0) {
            out[0] = c * ((double)S / D3);
            out[1] = h3 * V;
            out[2] = h3 * Cs;
            out[3] = (double)N;
        }
    }
}

// ------------------------------------------------------------- initial chi
__global__ void k_init_sphere(GridDesc g, float cx, float cy, float cz, float R,
                              uint8_t *__restrict__ chi)
{
    const long long nyz = (long long)g.ny * g.nz;
    const long long G = nyz * g.nx;
    const long long p = (long long)blockIdx.x * CT + threadIdx.x;
    if (p >= G) return;
    const int i = (int)(p / nyz);
    const long long rem = p - (long long)i * nyz;
    const int j = (int)(rem / g.nz);
    const int k = (int)(rem - (long long)j * g.nz);
    const float dx = cell_pos(i, g.cx, g.h) - cx;
    const float dy = cell_pos(j, g.cy, g.h) - cy;
    const float dz = cell_pos(k, g.cz, g.h) - cz;
    chi[p] = (sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) < R) ? 1 : 0;
}

// Tight start (Sec. 3.1, Initial surfaces): chi = 1 where min_i(|x - r_i| -
// d_i) < 0.  One block per tile of 4 x 8 x 8 cells: the block first keeps
// the atoms whose ball, widened by kTightMargin, reaches the tile's box
// (distance from the centre to the box at most d_i + margin), then every
// cell takes the minimum over those.  A discarded atom's |x - r_i| - d_i is
// at least the margin, far above the FP32 rounding of the distance, so it
// could not have made the minimum negative: the labels are those of the
// minimum over all atoms, in O(cells x nearby atoms) instead of O(cells x
// atoms).
constexpr int IT_X = 4, IT_Y = 8, IT_Z = 8;      // tile (IT_X * IT_Y * IT_Z = CT)
constexpr int IT_LIST = 1024;                     // atoms examined per pass
constexpr float kTightMargin = 1.0e-3f;           // Angstrom
static_assert(IT_X * IT_Y * IT_Z == CT, "one cell per thread");

static unsigned tight_blocks(const GridDesc &g)
{
    return (unsigned)(((g.nx + IT_X - 1) / IT_X) * ((g.ny + IT_Y - 1) / IT_Y) *
                      ((g.nz + IT_Z - 1) / IT_Z));
}

__global__ void __launch_bounds__(CT)
k_init_tight(GridDesc g, const float4 *__restrict__ xyzd, int n,
             uint8_t *__restrict__ chi)
{
    __shared__ float4 s_a[IT_LIST];
    __shared__ int s_cnt;
    const int ntz = (g.nz + IT_Z - 1) / IT_Z, nty = (g.ny + IT_Y - 1) / IT_Y;
    const int tz = blockIdx.x % ntz, ty = (blockIdx.x / ntz) % nty, tx = blockIdx.x / (ntz * nty);
    const int i0 = tx * IT_X, j0 = ty * IT_Y, k0 = tz * IT_Z;
    const int i = i0 + threadIdx.x / (IT_Y * IT_Z), j = j0 + (threadIdx.x / IT_Z) % IT_Y,
              k = k0 + threadIdx.x % IT_Z;
    const bool live = i < g.nx && j < g.ny && k < g.nz;
    const float x = cell_pos(i, g.cx, g.h), y = cell_pos(j, g.cy, g.h), z = cell_pos(k, g.cz, g.h);
    // the box of the tile's cells inside the grid
    const float lx = cell_pos(i0, g.cx, g.h), hx = cell_pos(min(i0 + IT_X, g.nx) - 1, g.cx, g.h);
    const float ly = cell_pos(j0, g.cy, g.h), hy = cell_pos(min(j0 + IT_Y, g.ny) - 1, g.cy, g.h);
    const float lz = cell_pos(k0, g.cz, g.h), hz = cell_pos(min(k0 + IT_Z, g.nz) - 1, g.cz, g.h);
    float phi = 3.0e38f;
    for (int base = 0; base < n; base += IT_LIST) {
        const int cnt = min(IT_LIST, n - base);
        __syncthreads();          // the previous list is no longer read
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += CT) {
            const float4 A = xyzd[base + m];
            const float gx = fmaxf(fmaxf(lx - A.x, A.x - hx), 0.f);
            const float gy = fmaxf(fmaxf(ly - A.y, A.y - hy), 0.f);
            const float gz = fmaxf(fmaxf(lz - A.z, A.z - hz), 0.f);
            const float reach = A.w + kTightMargin;
            if (reach > 0.f && fmaf(gx, gx, fmaf(gy, gy, gz * gz)) <= reach * reach)
                s_a[atomicAdd(&s_cnt, 1)] = A;
        }
        __syncthreads();
        const int c = s_cnt;
        for (int m = 0; m < c; ++m) {
            const float4 A = s_a[m];
            const float dx = x - A.x, dy = y - A.y, dz = z - A.z;
            phi = fminf(phi, sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) - A.w);
        }
    }
    if (live) chi[((long long)i * g.ny + j) * g.nz + k] = (phi < 0.f) ? 1 : 0;
}

// ------------------------------------------------------------- launchers
void launch_conv_z(const GridDesc &g, const KernelW &kw, const uint8_t *chi,
                   uint16_t *T1, cudaStream_t st)
{
    const Q17 w = centred(kw);
    const long long G = (long long)g.nx * g.ny * g.nz;
    count_launch();
    QPack qp;
    if (g.nz % 8 == 0 && (uintptr_t)chi % 8 == 0 && (uintptr_t)T1 % 16 == 0) {
        const unsigned nchunk = (unsigned)(G / 8);
        if (pack_dp4a(w, &qp))
            k_conv_z8_dp4a<<<(nchunk + CT - 1) / CT, CT, 0, st>>>(qp, chi, T1, g.nz, nchunk);
        else
            k_conv_z8<<<(nchunk + CT - 1) / CT, CT, 0, st>>>(w, chi, T1, g.nz, nchunk);
    } else {
        k_conv_z<<<cell_blocks(g), CT, 0, st>>>(g, w, chi, T1);
    }
}
void launch_conv_y(const GridDesc &g, const KernelW &kw, const uint16_t *T1,
                   uint32_t *T2, cudaStream_t st)
{
    const Q17 w = centred(kw);
    const long long nyz = (long long)g.ny * g.nz;
    if (VESIS_CONV_TILE && g.nx <= 65535)
        launch_tile(w, T1, T2, g.ny, g.nz, nyz, g.nx, g.nz, st);
    else if (g.nz % 2 == 0 && (uintptr_t)T1 % 4 == 0 && (uintptr_t)T2 % 8 == 0)
        launch_walk<2>(w, T1, T2, g.ny, g.nz, nyz, g.nx, g.nz, st);
    else
        launch_walk<1>(w, T1, T2, g.ny, g.nz, nyz, g.nx, g.nz, st);
}
void launch_conv_x(const GridDesc &g, const KernelW &kw, const uint32_t *T2,
                   uint32_t *W, cudaStream_t st)
{
    const Q17 w = centred(kw);
    const long long nyz = (long long)g.ny * g.nz;
    if (VESIS_CONV_TILE && g.ny <= 65535)
        launch_tile(w, T2, W, g.nx, nyz, g.nz, g.ny, g.nz, st);
    else if (g.nz % 2 == 0 && (uintptr_t)T2 % 8 == 0 && (uintptr_t)W % 8 == 0)
        launch_walk<2>(w, T2, W, g.nx, nyz, g.nz, g.ny, g.nz, st);
    else
        launch_walk<1>(w, T2, W, g.nx, nyz, g.nz, g.ny, g.nz, st);
}
void launch_conv3(const GridDesc &g, int R, const int *k3, const uint8_t *chi,
                  uint32_t *W, cudaStream_t st)
{
    const long long G = (long long)g.nx * g.ny * g.nz;
    count_launch();
    if (g.nz % 8 == 0 && (uintptr_t)chi % 8 == 0 && (uintptr_t)W % 16 == 0) {
        const unsigned nchunk = (unsigned)(G / 8);
        k_conv3_z8<<<(nchunk + CT - 1) / CT, CT, 0, st>>>(g.nx, g.ny, g.nz, R, k3, chi, W,
                                                            nchunk);
    } else {
        k_conv3<<<cell_blocks(g), CT, 0, st>>>(g, R, k3, chi, W);
    }
}
void launch_flip_energy(const GridDesc &g, const uint32_t *W,
                        const uint8_t *chi, const float *U, const FlipConst &fc,
                        double *dE, uint8_t *cand, cudaStream_t st)
{
    count_launch();
    k_flip_energy<<<cell_blocks(g), CT, 0, st>>>(g, W, chi, U, fc, dE, cand);
}
void launch_terms(const GridDesc &g, const uint8_t *chi, const uint32_t *W,
                  const float *U, const float *Ex, const float *Ey,
                  const float *Ez, float cfa, unsigned ksum, long long *part_s,
                  double *part_v, double *part_c, cudaStream_t st)
{
    const long long G = (long long)g.nx * g.ny * g.nz;
    count_launch();
    k_terms<<<terms_blocks(G), CT, 0, st>>>(g, chi, W, U, Ex, Ey, Ez, cfa, ksum,
                                            part_s, part_v, part_c);
}
void launch_terms_final(const long long *part_s, const double *part_v,
                        const double *part_c, int nb, double c, double D3,
                        double h3, double *out, cudaStream_t st)
{
    count_launch();
    k_terms_final<<<1, 1024, 0, st>>>(part_s, part_v, part_c, nb, c, D3, h3, out);
}
void launch_init_sphere(const GridDesc &g, float cx, float cy, float cz,
                        float radius, uint8_t *chi, cudaStream_t st)
{
    count_launch();
    k_init_sphere<<<cell_blocks(g), CT, 0, st>>>(g, cx, cy, cz, radius, chi);
}
void launch_init_tight(const GridDesc &g, const float4 *xyzd, int n,
                       uint8_t *chi, cudaStream_t st)
{
    count_launch();
    k_init_tight<<<tight_blocks(g), CT, 0, st>>>(g, xyzd, n, chi);
}

}  // namespace vesis
