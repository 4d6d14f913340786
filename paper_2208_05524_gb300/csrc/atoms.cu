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

// Solute-solute terms (Eq. Gss): harmonic bonds, and LJ plus Coulomb over
// the pairs not joined by a bond (mixing (s_i + s_j)/2, sqrt(e_i e_j)).
// Block (x, y) owns atoms i of tile x and visits the atoms j of chunk y, so
// each pair is counted twice and the energies are halved; bonds (a
// per-atom CSR list) are added by chunk 0 in FP64.  Per-chunk FP64 gradient
// partials are summed in chunk order afterwards.
//
// The pair terms run in double-float arithmetic: a value is the unevaluated
// sum hi + lo of two FP32 numbers (about 48 significant bits), built from
// the error-free transformations of Knuth (TwoSum) and Dekker (FastTwoSum,
// and the product's error recovered with one FMA).  The FP32 pipes do the
// work that FP64 would do at a small fraction of their rate.  Differences
// of coordinates use the accurate sum (error relative to the result), all
// other sums the short one (error relative to the operands); 1/r is FP32
// rsqrt refined by one Newton step whose residual 1 - r^2 y^2 is formed in
// double-float (relative error about 1.5 (2^-23)^2).  Each 128-atom stage's
// sums are added into FP64 accumulators, so the long sums stay in FP64.
constexpr int SS_THREADS = 128;
constexpr int SS_TILE = 128;
constexpr int kMaxExcl = 8;

SsPlan plan_ss(int n, int nsm)
{
    SsPlan sp;
    sp.tiles = (n + SS_THREADS - 1) / SS_THREADS;
    int nchunk = (8 * nsm + sp.tiles - 1) / sp.tiles;   // about 8 blocks per SM
    const int maxc = (n + 31) / 32;
    if (nchunk < 1) nchunk = 1;
    if (nchunk > maxc) nchunk = maxc;
    int len = (n + nchunk - 1) / nchunk;
    len = (len + 31) / 32 * 32;
    sp.chunk_len = len;
    sp.nchunk = (n + len - 1) / len;
    return sp;
}

struct dfl {
    float h, l;     // value = h + l, |l| <= ulp(h) / 2
};

__device__ __forceinline__ dfl df_of(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double df_val(dfl a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b with an error relative to |a| + |b|
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    const dfl s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

// a - b with an error relative to |a - b|
__device__ __forceinline__ dfl df_sub_acc(dfl a, dfl b)
{
    dfl s = two_sum(a.h, -b.h);
    const dfl t = two_sum(a.l, -b.l);
    s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_mulf(dfl a, float f)
{
    const float p = __fmul_rn(a.h, f);
    float e = __fmaf_rn(a.h, f, -p);
    e = __fmaf_rn(a.l, f, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ dfl df_sqr(dfl a)
{
    const float p = __fmul_rn(a.h, a.h);
    float e = __fmaf_rn(a.h, a.h, -p);
    e = __fmaf_rn(__fadd_rn(a.h, a.h), a.l, e);
    return fast_two_sum(p, e);
}

// exact scaling by a power of two
__device__ __forceinline__ dfl df_scale(dfl a, float p2) { return {a.h * p2, a.l * p2}; }

// 1 / sqrt(x): y0 = rsqrt(x.h), then y0 (1 + h / 2) with h = 1 - x y0^2
// formed in double-float (1 - t.h is exact, t.h being within a few ulp of 1)
__device__ __forceinline__ dfl df_rsqrt(dfl x)
{
    const float y = rsqrtf(x.h);
    const dfl t = df_mulf(df_mulf(x, y), y);
    const float h = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);
    return fast_two_sum(y, __fmul_rn(__fmul_rn(y, h), 0.5f));
}

__global__ void __launch_bounds__(SS_THREADS)
k_ss(const double *__restrict__ xyz, const double *__restrict__ sig,
     const double *__restrict__ sqeps, const double *__restrict__ q,
     const int *__restrict__ excl, const int *__restrict__ bond_ptr,
     const int *__restrict__ bond_other, const double *__restrict__ bond_k,
     const double *__restrict__ bond_r0, int n, int chunk_len, double coul,
     double *__restrict__ e_part, double *__restrict__ g_part)
{
    // staged atoms j as double-float: x, y, z, sigma / 2, sqrt(eps), q
    __shared__ __align__(16) dfl s_a[SS_TILE][6];
    __shared__ double s_red[3][SS_THREADS / 32];
    const int i = blockIdx.x * SS_THREADS + threadIdx.x;
    const bool live = i < n;
    const int jb = blockIdx.y * chunk_len;
    const int je = min(n, jb + chunk_len);
    double xi = 0, yi = 0, zi = 0;
    dfl Xi = {0.f, 0.f}, Yi = Xi, Zi = Xi, Si = Xi, Ei = Xi, Qi = Xi;
    int ex[kMaxExcl];
#pragma unroll
    for (int e = 0; e < kMaxExcl; ++e) ex[e] = -1;
    if (live) {
        xi = xyz[3 * i]; yi = xyz[3 * i + 1]; zi = xyz[3 * i + 2];
        Xi = df_of(xi); Yi = df_of(yi); Zi = df_of(zi);
        Si = df_of(0.5 * sig[i]);
        Ei = df_scale(df_of(sqeps[i]), 4.0f);     // 4 sqrt(eps_i): 4 eps_ij in one product
        Qi = df_of(coul * q[i]);
#pragma unroll
        for (int e = 0; e < kMaxExcl; ++e) ex[e] = excl[i * kMaxExcl + e];
    }
    double elj = 0.0, ec = 0.0, eb = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int base = jb; base < je; base += SS_TILE) {
        const int cnt = min(SS_TILE, je - base);
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += SS_THREADS) {
            const int j = base + m;
            s_a[m][0] = df_of(xyz[3 * j]);
            s_a[m][1] = df_of(xyz[3 * j + 1]);
            s_a[m][2] = df_of(xyz[3 * j + 2]);
            s_a[m][3] = df_of(0.5 * sig[j]);
            s_a[m][4] = df_of(sqeps[j]);
            s_a[m][5] = df_of(q[j]);
        }
        __syncthreads();
        if (!live) continue;
        const dfl z0 = {0.f, 0.f};
        dfl sl = z0, sc = z0, sx = z0, sy = z0, sz = z0;   // this stage's sums
        for (int m = 0; m < cnt; ++m) {
            const int j = base + m;
            bool skip = (j == i);
#pragma unroll
            for (int e = 0; e < kMaxExcl; ++e) skip |= (ex[e] == j);
            if (skip) continue;
            const dfl dx = df_sub_acc(Xi, s_a[m][0]);
            const dfl dy = df_sub_acc(Yi, s_a[m][1]);
            const dfl dz = df_sub_acc(Zi, s_a[m][2]);
            const dfl r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
            const dfl ir = df_rsqrt(r2);
            const dfl ir2 = df_sqr(ir);
            const dfl sg = df_add(Si, s_a[m][3]);
            const dfl ep4 = df_mul(Ei, s_a[m][4]);
            const dfl sr2 = df_mul(df_sqr(sg), ir2);
            const dfl sr6 = df_mul(df_sqr(sr2), sr2);
            const dfl sr12 = df_sqr(sr6);
            const dfl cq = df_mul(df_mul(Qi, s_a[m][5]), ir);
            sl = df_add(sl, df_mul(ep4, df_add(sr12, df_neg(sr6))));
            sc = df_add(sc, cq);
            // (dU/dr) / r = (4 eps (6 sr6 - 12 sr12) - cq) / r^2
            const dfl f = df_mul(df_add(df_mul(ep4, df_add(df_mulf(sr6, 6.0f),
                                                          df_mulf(sr12, -12.0f))),
                                        df_neg(cq)),
                                 ir2);
            sx = df_add(sx, df_mul(f, dx));
            sy = df_add(sy, df_mul(f, dy));
            sz = df_add(sz, df_mul(f, dz));
        }
        elj += df_val(sl);
        ec += df_val(sc);
        gx += df_val(sx);
        gy += df_val(sy);
        gz += df_val(sz);
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

// Sum of the blocks' partials, one warp per term: lane l adds blocks l,
// l + 32, ... in order, then the lanes' sums are combined by a fixed tree,
// so the result does not depend on timing.
__global__ void k_ss_final(const double *__restrict__ e_part, int nb, double *out3)
{
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += e_part[3 * b + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) out3[c] = t;
}

void launch_ss_final(const double *e_part, int nb, double *out3, cudaStream_t st)
{
    count_launch();
    k_ss_final<<<1, 96, 0, st>>>(e_part, nb, out3);
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
