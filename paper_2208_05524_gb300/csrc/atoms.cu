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

namespace vesis {

// ------------------------------------------------------ bends and torsions
// Bend (i, j, k): 1/2 B (theta - theta0)^2 with theta the angle between
// r_i - r_j and r_k - r_j; torsion (i, j, k, l): sum_n C_n [1 + cos(n tau
// - psi_n)] with tau the angle between u = q1 x q2 and v = q2 x q3, q1 =
// r_j - r_i, q2 = r_k - r_j, q3 = r_l - r_k (Eq. Gss).  Gradients as in the
// paper's appendix: B (theta - theta0) grad theta, and dW/dLambda grad
// Lambda for Lambda = cos tau (phases 0 or pi).  A bend with sin theta = 0
// adds no gradient; a torsion whose u or v vanishes adds nothing.

__device__ __forceinline__ void bend_term(const double *x, int i, int j, int k, double B,
                                          double t0, double &e, double gi[3], double gk[3])
{
    double a[3], b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a[c] = x[3 * i + c] - x[3 * j + c];
        b[c] = x[3 * k + c] - x[3 * j + c];
    }
    const double la = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double lb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    double cs = (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (la * lb);
    cs = fmin(1.0, fmax(-1.0, cs));
    const double th = acos(cs);
    const double d = th - t0;
    e = 0.5 * B * d * d;
    const double sn = sin(th);
#pragma unroll
    for (int c = 0; c < 3; ++c) gi[c] = gk[c] = 0.0;
    if (sn < 1e-12) return;
    const double f = B * d / sn;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        gi[c] = -f * (b[c] / (la * lb) - cs * a[c] / (la * la));
        gk[c] = -f * (a[c] / (la * lb) - cs * b[c] / (lb * lb));
    }
}

__device__ __forceinline__ void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Energy and the gradients of the four atoms (g[0..3][3]); false when
// degenerate.
__device__ __forceinline__ bool torsion_term(const double *x, const int *ijkl, const double *C,
                                             const double *psi, double &e, double g[4][3])
{
    const int i = ijkl[0], j = ijkl[1], k = ijkl[2], l = ijkl[3];
    double q1[3], q2[3], q3[3], u[3], v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        q1[c] = x[3 * j + c] - x[3 * i + c];
        q2[c] = x[3 * k + c] - x[3 * j + c];
        q3[c] = x[3 * l + c] - x[3 * k + c];
    }
    cross3(q1, q2, u);
    cross3(q2, q3, v);
    const double lu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double lv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    e = 0.0;
    if (lu * lv < 1e-24) return false;
    const double uv = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
    const double lam = fmin(1.0, fmax(-1.0, uv / (lu * lv)));
    const double tau = acos(lam);
    double cps[7];
#pragma unroll
    for (int n = 0; n < 7; ++n) {
        e += C[n] * (1.0 + cos(n * tau - psi[n]));
        cps[n] = cos(psi[n]);
    }
    // dW/dLambda = sum_n C_n cos(psi_n) T_n'(Lambda), T_n the Chebyshev
    // polynomials (cos n tau = T_n(cos tau)), T_n' = n U_{n-1}
    double dW = 0.0, Um1 = 0.0, U0 = 1.0;     // U_{-1} = 0, U_0 = 1
#pragma unroll
    for (int n = 1; n < 7; ++n) {
        dW += C[n] * cps[n] * n * U0;          // U0 holds U_{n-1}
        const double U1 = 2.0 * lam * U0 - Um1;
        Um1 = U0;
        U0 = U1;
    }
    double du[3], dv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        du[c] = (v[c] * lu * lu - uv * u[c]) / (lu * lu * lu * lv);
        dv[c] = (u[c] * lv * lv - uv * v[c]) / (lu * lv * lv * lv);
    }
    double d1[3], d2a[3], d2b[3], d3[3];
    cross3(q2, du, d1);
    cross3(du, q1, d2a);
    cross3(q3, dv, d2b);
    cross3(dv, q2, d3);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double d2 = d2a[c] + d2b[c];
        g[0][c] = -dW * d1[c];
        g[1][c] = dW * (d1[c] - d2);
        g[2][c] = dW * (d2 - d3[c]);
        g[3][c] = dW * d3[c];
    }
    return true;
}

__global__ void k_bonded_energy(BondedDev b, const double *__restrict__ x,
                                double *__restrict__ part)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < b.nang) {
        double e, gi[3], gk[3];
        bend_term(x, b.ang[3 * m], b.ang[3 * m + 1], b.ang[3 * m + 2], b.angB[m], b.angT0[m], e,
                  gi, gk);
        part[m] = e;
    } else if (m < b.nang + b.ntor) {
        const int t = m - b.nang;
        double e, g[4][3];
        torsion_term(x, b.tor + 4 * t, b.torC + 7 * t, b.torPsi + 7 * t, e, g);
        part[m] = e;
    }
}

// grad[n] += the bend and torsion gradients of atom n, its terms in
// increasing order (no atomics: the sums are reproducible).
__global__ void k_bonded_grad(BondedDev b, const double *__restrict__ x, int n,
                              double *__restrict__ grad)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int e = b.ang_ptr[a]; e < b.ang_ptr[a + 1]; ++e) {
        const int m = b.ang_inc[e] >> 2, role = b.ang_inc[e] & 3;
        double en, gi[3], gk[3];
        bend_term(x, b.ang[3 * m], b.ang[3 * m + 1], b.ang[3 * m + 2], b.angB[m], b.angT0[m],
                  en, gi, gk);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            s[c] += role == 0 ? gi[c] : role == 2 ? gk[c] : -(gi[c] + gk[c]);
    }
    for (int e = b.tor_ptr[a]; e < b.tor_ptr[a + 1]; ++e) {
        const int t = b.tor_inc[e] >> 2, role = b.tor_inc[e] & 3;
        double en, g[4][3];
        if (!torsion_term(x, b.tor + 4 * t, b.torC + 7 * t, b.torPsi + 7 * t, en, g)) continue;
#pragma unroll
        for (int c = 0; c < 3; ++c) s[c] += g[role][c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) grad[3 * a + c] += s[c];
}

void launch_bonded(const BondedDev &b, const double *xyz, int n, double *part, double *e_bend,
                   double *e_tors, double *grad, cudaStream_t st)
{
    const int nt = b.nang + b.ntor;
    if (nt > 0) {
        count_launch();
        k_bonded_energy<<<(nt + 127) / 128, 128, 0, st>>>(b, xyz, part);
    }
    launch_sum_doubles(part, b.nang, e_bend, 0, st);
    launch_sum_doubles(part + b.nang, b.ntor, e_tors, 0, st);
    if (grad && nt > 0) {
        count_launch();
        k_bonded_grad<<<(n + 127) / 128, 128, 0, st>>>(b, xyz, n, grad);
    }
}

}  // namespace vesis
