// Per-atom kernels: FP32 packing of the atom data, the solute-solute terms
// of Eq. (Gss) and the adaptive-mobility step (Eq. moveatoms/adjustmml).
#include "vesis_internal.cuh"

namespace vesis {

__global__ void k_pack_atoms(const double *__restrict__ xyz, const double *centre,
                             const double *__restrict__ sig,
                             const double *__restrict__ eps,
                             const double *__restrict__ q, int n, double rho,
                             double cfa, float4 *__restrict__ xyzq,
                             float2 *__restrict__ ab, float4 *__restrict__ fcoef,
                             int *oob, const double *lo, const double *hi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const bool inside = x > lo[0] && x < hi[0] && y > lo[1] && y < hi[1] &&
                        z > lo[2] && z < hi[2];
    if (!inside) atomicOr(oob, 1);
    const double s2 = sig[i] * sig[i];
    const double s6 = s2 * s2 * s2;
    const double A = 4.0 * eps[i] * s6 * s6;
    const double B = 4.0 * eps[i] * s6;
    xyzq[i] = make_float4((float)(x - centre[0]), (float)(y - centre[1]),
                          (float)(z - centre[2]), (float)q[i]);
    ab[i] = make_float2((float)A, (float)B);
    fcoef[i] = make_float4((float)(12.0 * rho * A), (float)(-6.0 * rho * B),
                           (float)(-2.0 * cfa * q[i]), 0.f);
}

void launch_pack_atoms(const double *xyz, const double *centre,
                       const double *sig, const double *eps, const double *q,
                       int n, double rho, double cfa, float4 *xyzq,
                       float2 *ab, float4 *fcoef, int *oob, const double *lo,
                       const double *hi, cudaStream_t st)
{
    count_launch();
    k_pack_atoms<<<(n + 127) / 128, 128, 0, st>>>(xyz, centre, sig, eps, q, n,
                                                  rho, cfa, xyzq, ab, fcoef,
                                                  oob, lo, hi);
}

// Solute-solute terms in FP64: harmonic bonds, and LJ plus Coulomb over the
// pairs not joined by a bond (mixing (s_i + s_j)/2, sqrt(e_i e_j)).  Block
// (x, y) owns atoms i of tile x and visits the atoms j of chunk y, so each
// pair is counted twice and the energies are halved; bonds (a per-atom CSR
// list) are added by chunk 0.  Per-chunk FP64 gradient partials are summed
// in chunk order afterwards.  1/r comes from an FP32 reciprocal square root
// refined by two Newton-Raphson steps y <- y (3/2 - r^2 y^2 / 2), which
// reaches double precision without a double divide or square root.
constexpr int SS_THREADS = 128;
constexpr int SS_TILE = 128;
constexpr int kMaxExcl = 8;

SsPlan plan_ss(int n, int nsm)
{
    SsPlan sp;
    sp.tiles = (n + SS_THREADS - 1) / SS_THREADS;
    int nchunk = (2 * nsm + sp.tiles - 1) / sp.tiles;
    const int maxc = (n + 31) / 32;
    if (nchunk < 1) nchunk = 1;
    if (nchunk > maxc) nchunk = maxc;
    int len = (n + nchunk - 1) / nchunk;
    len = (len + 31) / 32 * 32;
    sp.chunk_len = len;
    sp.nchunk = (n + len - 1) / len;
    return sp;
}

__device__ __forceinline__ double inv_sqrt_d(double r2)
{
    double y = (double)rsqrtf((float)r2);
    y = y * (1.5 - 0.5 * r2 * y * y);
    y = y * (1.5 - 0.5 * r2 * y * y);
    return y;
}

__global__ void __launch_bounds__(SS_THREADS)
k_ss(const double *__restrict__ xyz, const double *__restrict__ sig,
     const double *__restrict__ sqeps, const double *__restrict__ q,
     const int *__restrict__ excl, const int *__restrict__ bond_ptr,
     const int *__restrict__ bond_other, const double *__restrict__ bond_k,
     const double *__restrict__ bond_r0, int n, int chunk_len, double coul,
     double *__restrict__ e_part, double *__restrict__ g_part)
{
    __shared__ double s_x[SS_TILE], s_y[SS_TILE], s_z[SS_TILE];
    __shared__ double s_s[SS_TILE], s_e[SS_TILE], s_q[SS_TILE];
    __shared__ double s_red[3][SS_THREADS / 32];
    const int i = blockIdx.x * SS_THREADS + threadIdx.x;
    const bool live = i < n;
    const int jb = blockIdx.y * chunk_len;
    const int je = min(n, jb + chunk_len);
    double xi = 0, yi = 0, zi = 0, si = 0, ei = 0, qi = 0;
    int ex[kMaxExcl];
#pragma unroll
    for (int e = 0; e < kMaxExcl; ++e) ex[e] = -1;
    if (live) {
        xi = xyz[3 * i]; yi = xyz[3 * i + 1]; zi = xyz[3 * i + 2];
        si = sig[i]; ei = sqeps[i]; qi = q[i];
#pragma unroll
        for (int e = 0; e < kMaxExcl; ++e) ex[e] = excl[i * kMaxExcl + e];
    }
    double elj = 0.0, ec = 0.0, eb = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int base = jb; base < je; base += SS_TILE) {
        const int cnt = min(SS_TILE, je - base);
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += SS_THREADS) {
            const int j = base + m;
            s_x[m] = xyz[3 * j]; s_y[m] = xyz[3 * j + 1]; s_z[m] = xyz[3 * j + 2];
            s_s[m] = sig[j]; s_e[m] = sqeps[j]; s_q[m] = q[j];
        }
        __syncthreads();
        if (!live) continue;
        for (int m = 0; m < cnt; ++m) {
            const int j = base + m;
            bool skip = (j == i);
#pragma unroll
            for (int e = 0; e < kMaxExcl; ++e) skip |= (ex[e] == j);
            if (skip) continue;
            const double dx = xi - s_x[m], dy = yi - s_y[m], dz = zi - s_z[m];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double ir = inv_sqrt_d(r2);
            const double ir2 = ir * ir;
            const double s = 0.5 * (si + s_s[m]);
            const double ep = ei * s_e[m];
            const double sr2 = s * s * ir2;
            const double sr6 = sr2 * sr2 * sr2;
            const double cq = coul * qi * s_q[m] * ir;
            elj += 4.0 * ep * (sr6 * sr6 - sr6);
            ec += cq;
            // (dU/dr)/r
            const double f = (4.0 * ep * (-12.0 * sr6 * sr6 + 6.0 * sr6) - cq) * ir2;
            gx += f * dx;
            gy += f * dy;
            gz += f * dz;
        }
    }
    if (live) {
        if (blockIdx.y == 0) {
            for (int b = bond_ptr[i]; b < bond_ptr[i + 1]; ++b) {
                const int j = bond_other[b];
                const double dx = xi - xyz[3 * j], dy = yi - xyz[3 * j + 1],
                             dz = zi - xyz[3 * j + 2];
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                const double dr = r - bond_r0[b];
                eb += 0.5 * bond_k[b] * dr * dr;
                const double f = bond_k[b] * dr / r;
                gx += f * dx;
                gy += f * dy;
                gz += f * dz;
            }
        }
        double *o = g_part + ((long long)blockIdx.y * n + i) * 3;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
    }
    double v[3] = {0.5 * eb, 0.5 * elj, 0.5 * ec};
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
        if (l == 0) s_red[c][w] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        for (int c = 0; c < 3; ++c) {
            double t = 0.0;
            for (int q2 = 0; q2 < SS_THREADS / 32; ++q2) t += s_red[c][q2];
            e_part[3 * blk + c] = t;
        }
    }
}

void launch_ss(const SsPlan &sp, const double *xyz, const double *sig,
               const double *sqeps, const double *q, const int *excl,
               const int *bond_ptr, const int *bond_other, const double *bond_k,
               const double *bond_r0, int n, double coul, double *e_part,
               double *g_part, cudaStream_t st)
{
    count_launch();
    k_ss<<<dim3(sp.tiles, sp.nchunk), SS_THREADS, 0, st>>>(
        xyz, sig, sqeps, q, excl, bond_ptr, bond_other, bond_k, bond_r0, n,
        sp.chunk_len, coul, e_part, g_part);
}

__global__ void k_ss_final(const double *__restrict__ e_part, int nb, double *out3)
{
    double t[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b)
        for (int c = 0; c < 3; ++c) t[c] += e_part[3 * b + c];
    out3[0] = t[0];
    out3[1] = t[1];
    out3[2] = t[2];
}

void launch_ss_final(const double *e_part, int nb, double *out3, cudaStream_t st)
{
    count_launch();
    k_ss_final<<<1, 1, 0, st>>>(e_part, nb, out3);
}

// grad = a + b and max |grad component| (non-negative doubles order like
// their bit patterns, so an integer max is exact and order-independent).
__global__ void k_grad_combine(const double *__restrict__ a,
                               const double *__restrict__ b,
                               double *__restrict__ grad, int n3,
                               unsigned long long *gmax_bits)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double m = 0.0;
    if (t < n3) {
        const double g = a[t] + b[t];
        grad[t] = g;
        m = fabs(g);
        if (!(m == m) || m > 1.0e300) m = 1.0e308;   // NaN / inf -> huge
    }
    unsigned long long bits = __double_as_longlong(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_down_sync(0xffffffffu, bits, o);
        bits = ob > bits ? ob : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(gmax_bits, bits);
}

void launch_grad_combine(const double *a, const double *b, double *grad,
                         int n3, unsigned long long *gmax_bits, cudaStream_t st)
{
    cudaMemsetAsync(gmax_bits, 0, sizeof(unsigned long long), st);
    count_launch();
    k_grad_combine<<<(n3 + 255) / 256, 256, 0, st>>>(a, b, grad, n3, gmax_bits);
}

__global__ void k_mobility(const double *__restrict__ xyz,
                           const double *__restrict__ grad,
                           const unsigned long long *gmax_bits,
                           const double *M, double *__restrict__ xyz_new, int n3)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3) return;
    const double gmax = __longlong_as_double((long long)*gmax_bits);
    const double step = (gmax > 0.0) ? (*M / gmax) : 0.0;
    xyz_new[t] = xyz[t] - step * grad[t];
}

void launch_mobility(const double *xyz, const double *grad,
                     const unsigned long long *gmax_bits, const double *M,
                     double *xyz_new, int n3, cudaStream_t st)
{
    count_launch();
    k_mobility<<<(n3 + 255) / 256, 256, 0, st>>>(xyz, grad, gmax_bits, M,
                                                xyz_new, n3);
}

}  // namespace vesis
