/*
 * Plain FP64 CPU oracle for the VESIS hot path (Liu, Zhang, Cheng, Li,
 * arXiv 2208.05524).  TEST INFRASTRUCTURE ONLY: tests, the smoke check and
 * the CPU-baseline leg of the benchmark call it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Every routine is a direct loop over the definition it cites; there is no
 * blocking, fusion or reordering beyond what the definition states.  Outer
 * loops over independent outputs carry an OpenMP pragma.
 *
 * Grid: n[0] x n[1] x n[2] cells, spacing h, cell centres at
 * origin + (i + 1/2) h (Sec. 3.1), linear index (i*ny + j)*nz + k.
 *
 * Compile with -ffp-contract=off: the flip-energy test (Eq. dGj1/dGj2) must
 * round exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, k) (((int64_t)(i) * ny + (j)) * nz + (k))

/* ------------------------------------------------------------------ pairs
 * Energy density of Eq. (Ur): U(x) = rho_w sum_i U_LJ^(i)(|x - r_i|)
 *   + C |sum_i Q_i (x - r_i)/|x - r_i|^3|^2,
 * U_LJ(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] (Eq. LJpotential).
 * The distance is clamped, r = max(|x - r_i|, rmin), identically in every
 * pair term.  Output per point: lj = sum_i U_LJ^(i) (without rho_w) and the
 * Coulomb field E = sum_i Q_i d / r^3, d = x - r_i.
 */
static void point_terms(const double x[3], int na, const double *xyz,
                        const double *sig, const double *eps, const double *q,
                        double rmin, double *lj_out, double E_out[3])
{
    double lj = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int a = 0; a < na; ++a) {
        double dx = x[0] - xyz[3 * a + 0];
        double dy = x[1] - xyz[3 * a + 1];
        double dz = x[2] - xyz[3 * a + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r < rmin) r = rmin;
        double sr = sig[a] / r;
        double sr6 = sr * sr * sr * sr * sr * sr;
        lj += 4.0 * eps[a] * (sr6 * sr6 - sr6);
        double r3 = r * r * r;
        ex += q[a] * dx / r3;
        ey += q[a] * dy / r3;
        ez += q[a] * dz / r3;
    }
    *lj_out = lj;
    E_out[0] = ex;
    E_out[1] = ey;
    E_out[2] = ez;
}

void or_grid_terms(int nx, int ny, int nz, double h, const double *origin,
                   int na, const double *xyz, const double *sig,
                   const double *eps, const double *q, double rmin,
                   double *lj, double *E /* G x 3 */)
{
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                double x[3] = {origin[0] + (i + 0.5) * h,
                               origin[1] + (j + 0.5) * h,
                               origin[2] + (k + 0.5) * h};
                int64_t p = IDX(i, j, k);
                point_terms(x, na, xyz, sig, eps, q, rmin, &lj[p], &E[3 * p]);
            }
}

void or_point_terms(int64_t np, const double *pts, int na, const double *xyz,
                    const double *sig, const double *eps, const double *q,
                    double rmin, double *lj, double *E)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < np; ++p)
        point_terms(&pts[3 * p], na, xyz, sig, eps, q, rmin, &lj[p], &E[3 * p]);
}

/* Gradient with respect to atom n of the volume term
 *   sum_x wt(x) U(x)   (grid: wt = h^3 on solvent cells, 0 on solute;
 *                       far field: quadrature weights),
 * from differentiating Eq. (Ur) exactly (the appendix formula, Eq.
 * GradientG, keeps only part of the Coulomb-field derivative):
 *   d/dr_n [rho_w U_LJ(|d|)] = -rho_w U_LJ'(r) d / r
 *   d/dr_n [C |E|^2]         = -2 C Q_n [E / r^3 - 3 (d.E) d / r^5]
 * with d = x - r_n.  Where r is clamped to rmin the LJ term is constant
 * (zero derivative) and the field term is Q_n d / rmin^3, whose derivative
 * drops the d d^T part.
 */
static void atom_grad(const double a[3], double sig, double eps, double qn,
                      const double x[3], const double E[3], double wt,
                      double rho_w, double C, double rmin, double g[3])
{
    double d[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    int clamped = r < rmin;
    double re = clamped ? rmin : r;
    double re3 = re * re * re;
    double dE = d[0] * E[0] + d[1] * E[1] + d[2] * E[2];
    double dUdr = 0.0;
    if (!clamped) {
        double sr = sig / r;
        double sr6 = sr * sr * sr * sr * sr * sr;
        dUdr = 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r;
    }
    for (int l = 0; l < 3; ++l) {
        double glj = clamped ? 0.0 : -rho_w * dUdr * d[l] / r;
        double gfield = E[l] / re3;
        if (!clamped) gfield -= 3.0 * dE * d[l] / (re3 * re * re);
        g[l] += wt * (glj - 2.0 * C * qn * gfield);
    }
}

void or_grid_grad(int nx, int ny, int nz, double h, const double *origin,
                  const uint8_t *chi, const double *E, int na,
                  const double *xyz, const double *sig, const double *eps,
                  const double *q, double rho_w, double C, double rmin,
                  double *grad /* na x 3 */)
{
    double h3 = h * h * h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < na; ++n) {
        double g[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < nx; ++i)
            for (int j = 0; j < ny; ++j)
                for (int k = 0; k < nz; ++k) {
                    int64_t p = IDX(i, j, k);
                    if (chi[p]) continue;
                    double x[3] = {origin[0] + (i + 0.5) * h,
                                   origin[1] + (j + 0.5) * h,
                                   origin[2] + (k + 0.5) * h};
                    atom_grad(&xyz[3 * n], sig[n], eps[n], q[n], x, &E[3 * p],
                              h3, rho_w, C, rmin, g);
                }
        grad[3 * n + 0] = g[0];
        grad[3 * n + 1] = g[1];
        grad[3 * n + 2] = g[2];
    }
}

void or_point_grad(int64_t np, const double *pts, const double *wts,
                   const double *E, int na, const double *xyz,
                   const double *sig, const double *eps, const double *q,
                   double rho_w, double C, double rmin, double *grad)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < na; ++n) {
        double g[3] = {0.0, 0.0, 0.0};
        for (int64_t p = 0; p < np; ++p)
            atom_grad(&xyz[3 * n], sig[n], eps[n], q[n], &pts[3 * p], &E[3 * p],
                      wts[p], rho_w, C, rmin, g);
        grad[3 * n + 0] = g[0];
        grad[3 * n + 1] = g[1];
        grad[3 * n + 2] = g[2];
    }
}

/* ---------------------------------------------------------- solute-solute
 * G_ss of Eq. (Gss): harmonic bonds 1/2 A (r - r0)^2, plus LJ and Coulomb
 * over the non-bonded pairs (all pairs not joined by a bond).  Angle and
 * torsion terms are not part of these solutes.  Pair parameters mix as
 * sigma_ij = (sigma_i + sigma_j)/2, eps_ij = sqrt(eps_i eps_j); Coulomb is
 * lB Q_i Q_j / (eps_ss r) in kBT with lB the Bjerrum length.
 * Output: e[0] bonds, e[1] LJ, e[2] Coulomb; grad accumulates dG_ss/dr.
 */
static int bonded(int i, int j, int nb, const int *bonds)
{
    for (int b = 0; b < nb; ++b)
        if ((bonds[2 * b] == i && bonds[2 * b + 1] == j) ||
            (bonds[2 * b] == j && bonds[2 * b + 1] == i))
            return 1;
    return 0;
}

void or_ss(int na, const double *xyz, const double *sig, const double *eps,
           const double *q, int nb, const int *bonds, const double *bk,
           const double *br0, double coul, double *e, double *grad)
{
    double eb = 0.0, elj = 0.0, ec = 0.0;
    for (int n = 0; n < 3 * na; ++n) grad[n] = 0.0;
    for (int b = 0; b < nb; ++b) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1],
                       xyz[3 * i + 2] - xyz[3 * j + 2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        eb += 0.5 * bk[b] * (r - br0[b]) * (r - br0[b]);
        for (int l = 0; l < 3; ++l) {
            double f = bk[b] * (r - br0[b]) * d[l] / r;
            grad[3 * i + l] += f;
            grad[3 * j + l] -= f;
        }
    }
    for (int i = 0; i < na; ++i)
        for (int j = i + 1; j < na; ++j) {
            if (bonded(i, j, nb, bonds)) continue;
            double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1],
                           xyz[3 * i + 2] - xyz[3 * j + 2]};
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double s = 0.5 * (sig[i] + sig[j]);
            double ep = sqrt(eps[i] * eps[j]);
            double sr = s / r;
            double sr6 = sr * sr * sr * sr * sr * sr;
            elj += 4.0 * ep * (sr6 * sr6 - sr6);
            ec += coul * q[i] * q[j] / r;
            double dUdr = 4.0 * ep * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r
                          - coul * q[i] * q[j] / (r * r);
            for (int l = 0; l < 3; ++l) {
                double f = dUdr * d[l] / r;
                grad[3 * i + l] += f;
                grad[3 * j + l] -= f;
            }
        }
    e[0] = eb;
    e[1] = elj;
    e[2] = ec;
}

/* ------------------------------------------------------------- surface
 * Surface energy with the product (Gaussian) kernel in place of sin^2
 * (Eq. Area / Eq. 4flip):  E_s = c sum_{j solute} sum_{k solvent} g_jk,
 * g_jk = qa qb qc / D^3 for offsets (a,b,c) in [-r, r]^3, D = sum_a q_a.
 * Cells outside the box are solvent.  With w = g * chi (zero padding),
 * sum_k g_jk (1 - chi_k) = 1 - w_j, so E_s = c sum_j chi_j (1 - w_j).
 *
 * W = D^3 w is an exact integer: the convolution is done in three 1-D
 * passes along z, y, x (the kernel is a product), in int64.
 */
void or_conv(int nx, int ny, int nz, const uint8_t *chi, int r, const int *qw,
             int64_t *W)
{
    int64_t G = (int64_t)nx * ny * nz;
    int64_t *t1 = (int64_t *)malloc(sizeof(int64_t) * G);
    int64_t *t2 = (int64_t *)malloc(sizeof(int64_t) * G);
#pragma omp parallel for collapse(2)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t s = 0;
                for (int a = -r; a <= r; ++a)
                    if (k + a >= 0 && k + a < nz) s += (int64_t)qw[a + r] * chi[IDX(i, j, k + a)];
                t1[IDX(i, j, k)] = s;
            }
#pragma omp parallel for collapse(2)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t s = 0;
                for (int b = -r; b <= r; ++b)
                    if (j + b >= 0 && j + b < ny) s += (int64_t)qw[b + r] * t1[IDX(i, j + b, k)];
                t2[IDX(i, j, k)] = s;
            }
#pragma omp parallel for collapse(2)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t s = 0;
                for (int c = -r; c <= r; ++c)
                    if (i + c >= 0 && i + c < nx) s += (int64_t)qw[c + r] * t2[IDX(i + c, j, k)];
                W[IDX(i, j, k)] = s;
            }
    free(t1);
    free(t2);
}

/* Direct 3-D convolution with a full integer stencil k3 of (2r+1)^3
 * weights (offset (a,b,c) at ((a+r)(2r+1) + b+r)(2r+1) + c+r), zero
 * padding: the sin^2 kernel of Sec. 3.1 is not a product of 1-D factors. */
void or_conv3(int nx, int ny, int nz, const uint8_t *chi, int r, const int64_t *k3,
              int64_t *W)
{
    const int w = 2 * r + 1;
#pragma omp parallel for collapse(2)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t s = 0;
                for (int a = -r; a <= r; ++a) {
                    if (i + a < 0 || i + a >= nx) continue;
                    for (int b = -r; b <= r; ++b) {
                        if (j + b < 0 || j + b >= ny) continue;
                        for (int c = -r; c <= r; ++c) {
                            if (k + c < 0 || k + c >= nz) continue;
                            s += k3[((a + r) * w + (b + r)) * w + (c + r)] *
                                 chi[IDX(i + a, j + b, k + c)];
                        }
                    }
                }
                W[IDX(i, j, k)] = s;
            }
}

/* W of either kernel: the 1-D factors qw when k3 is NULL, else the stencil. */
static void conv_any(int nx, int ny, int nz, const uint8_t *chi, int r, const int *qw,
                     const int64_t *k3, int64_t *W)
{
    if (k3) or_conv3(nx, ny, nz, chi, r, k3, W);
    else or_conv(nx, ny, nz, chi, r, qw, W);
}

/* sum_j chi_j (S - W_j), exact; S = sum of all kernel weights (D^3 for the
 * product kernel).  E_s = c_N * this. */
int64_t or_surface_sum(int64_t G, const uint8_t *chi, const int64_t *W,
                       int64_t S)
{
    int64_t s = 0;
    for (int64_t p = 0; p < G; ++p)
        if (chi[p]) s += S - W[p];
    return s;
}

/* Candidates: cells next to the interface, i.e. with a face neighbour of
 * the opposite label; a neighbour outside the box counts as solvent. */
static int is_candidate(int nx, int ny, int nz, const uint8_t *chi, int i,
                        int j, int k)
{
    int c = chi[IDX(i, j, k)];
    const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                           {0, 1, 0},  {0, 0, -1}, {0, 0, 1}};
    for (int f = 0; f < 6; ++f) {
        int a = i + off[f][0], b = j + off[f][1], d = k + off[f][2];
        int nb = (a < 0 || a >= nx || b < 0 || b >= ny || d < 0 || d >= nz)
                     ? 0 : chi[IDX(a, b, d)];
        if (nb != c) return 1;
    }
    return 0;
}

/* Energy change of flipping cell j (Eq. dGj1 / dGj2 with the h^3 of the
 * centre-point rule restored):  with s = +1 for solvent -> solute and -1
 * for solute -> solvent, w_j = W_j / S and g0 = k0 / S (k0 the kernel's
 * centre weight),
 *   dE = c [ s (1 - 2 w_j) - g0 ] - s h^3 U_j.
 * With c_N = c / S the bracket times c is c_N N for the exact integer
 * N = s (S - 2 W_j) - k0, so dE = c_N N - s h^3 U: one rounded product for
 * each term and one rounded difference.  (For the Gaussian, S = 2^24 and
 * every step of c [s (1 - 2w) - g0] before the product with c is exact, so
 * the two forms agree bit for bit.) */
static double flip_energy(uint8_t chi_j, int64_t Wj, double U, double cN, int64_t S,
                          int64_t k0, double h3)
{
    double s = chi_j ? -1.0 : 1.0;
    int64_t N = (chi_j ? -(S - 2 * Wj) : (S - 2 * Wj)) - k0;
    double t1 = cN * (double)N;
    double t2 = h3 * U;
    return t1 - s * t2;
}

void or_delta_e(int nx, int ny, int nz, const uint8_t *chi, const int64_t *W,
                const double *U, double cN, int64_t S, int64_t k0, double h3,
                double *dE, uint8_t *cand)
{
#pragma omp parallel for collapse(2)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t p = IDX(i, j, k);
                cand[p] = (uint8_t)is_candidate(nx, ny, nz, chi, i, j, k);
                dE[p] = cand[p] ? flip_energy(chi[p], W[p], U[p], cN, S, k0, h3) : 0.0;
            }
}

/* ----------------------------------------------------- parallel flip rule
 * Data-parallel form of the min-heap flipping (Sec. 3.1, Step 2.2).  Every
 * candidate whose flip lowers the energy (dE < 0, FP64) gets the key
 * (order-preserving bits of (float)dE) << 32 | linear index; a smaller key
 * comes first in the heap's order (ties of float(dE) go to the smaller
 * index).  The grid is cut into bricks of edge B (B = 4 when r >= 3, else
 * 2) aligned at index 0; each brick's leader is its cell with the smallest
 * key.  A leader flips when no other brick's leader within Chebyshev
 * distance r has a smaller key.  Two flipped cells are therefore more than
 * r apart, the kernel couples none of them, and the energy change of the
 * round is exactly the sum of their dE.  The heap's top (the global
 * smallest key) always flips.
 *
 * or_select_cells is the finer rule "smallest key over the whole cube of
 * half-width r"; every cell it selects the brick rule selects too.  Tests
 * use it to check that relation.
 */
static uint64_t flip_key(double dE, int64_t p)
{
    float f = (float)dE;
    uint32_t u;
    memcpy(&u, &f, 4);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((uint64_t)u << 32) | (uint64_t)p;
}

int or_brick_edge(int r) { return r >= 3 ? 4 : 2; }

static void make_keys(int64_t G, const uint8_t *cand, const double *dE, uint64_t *keys)
{
#pragma omp parallel for
    for (int64_t p = 0; p < G; ++p)
        keys[p] = (cand[p] && dE[p] < 0.0) ? flip_key(dE[p], p) : UINT64_MAX;
}

int64_t or_select(int nx, int ny, int nz, const uint8_t *cand,
                  const double *dE, int r, uint8_t *sel, uint64_t *keys)
{
    int64_t G = (int64_t)nx * ny * nz;
    const int B = or_brick_edge(r);
    const int bx = (nx + B - 1) / B, by = (ny + B - 1) / B, bz = (nz + B - 1) / B;
    const int64_t NB = (int64_t)bx * by * bz;
    uint64_t *lead = (uint64_t *)malloc(sizeof(uint64_t) * NB);
    make_keys(G, cand, dE, keys);
    /* leaders: the smallest key of each brick */
#pragma omp parallel for collapse(2)
    for (int a = 0; a < bx; ++a)
        for (int b = 0; b < by; ++b)
            for (int c = 0; c < bz; ++c) {
                uint64_t m = UINT64_MAX;
                for (int i = a * B; i < a * B + B && i < nx; ++i)
                    for (int j = b * B; j < b * B + B && j < ny; ++j)
                        for (int k = c * B; k < c * B + B && k < nz; ++k)
                            if (keys[IDX(i, j, k)] < m) m = keys[IDX(i, j, k)];
                lead[((int64_t)a * by + b) * bz + c] = m;
            }
    for (int64_t p = 0; p < G; ++p) sel[p] = 0;
    int64_t nsel = 0;
#pragma omp parallel for collapse(2) reduction(+ : nsel)
    for (int a = 0; a < bx; ++a)
        for (int b = 0; b < by; ++b)
            for (int c = 0; c < bz; ++c) {
                const uint64_t m = lead[((int64_t)a * by + b) * bz + c];
                if (m == UINT64_MAX) continue;
                const int64_t p = (int64_t)(m & 0xffffffffu);
                const int i = (int)(p / ((int64_t)ny * nz)), j = (int)((p / nz) % ny),
                          k = (int)(p % nz);
                int best = 1;
                /* every brick that holds a cell of the cube around p */
                for (int a2 = (i - r < 0 ? 0 : i - r) / B; best && a2 <= (i + r < nx ? i + r : nx - 1) / B; ++a2)
                    for (int b2 = (j - r < 0 ? 0 : j - r) / B; best && b2 <= (j + r < ny ? j + r : ny - 1) / B; ++b2)
                        for (int c2 = (k - r < 0 ? 0 : k - r) / B; c2 <= (k + r < nz ? k + r : nz - 1) / B; ++c2) {
                            if (a2 == a && b2 == b && c2 == c) continue;
                            const uint64_t m2 = lead[((int64_t)a2 * by + b2) * bz + c2];
                            if (m2 >= m) continue;
                            const int64_t p2 = (int64_t)(m2 & 0xffffffffu);
                            const int i2 = (int)(p2 / ((int64_t)ny * nz)),
                                      j2 = (int)((p2 / nz) % ny), k2 = (int)(p2 % nz);
                            if (abs(i2 - i) <= r && abs(j2 - j) <= r && abs(k2 - k) <= r) {
                                best = 0;
                                break;
                            }
                        }
                if (best) {
                    sel[p] = 1;
                    nsel += 1;
                }
            }
    free(lead);
    return nsel;
}

int64_t or_select_cells(int nx, int ny, int nz, const uint8_t *cand,
                        const double *dE, int r, uint8_t *sel, uint64_t *keys)
{
    int64_t G = (int64_t)nx * ny * nz;
    make_keys(G, cand, dE, keys);
    int64_t nsel = 0;
#pragma omp parallel for collapse(2) reduction(+ : nsel)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t p = IDX(i, j, k);
                sel[p] = 0;
                uint64_t kp = keys[p];
                if (kp == UINT64_MAX) continue;
                int best = 1;
                for (int a = i - r; a <= i + r && best; ++a) {
                    if (a < 0 || a >= nx) continue;
                    for (int b = j - r; b <= j + r && best; ++b) {
                        if (b < 0 || b >= ny) continue;
                        for (int d = k - r; d <= k + r; ++d) {
                            if (d < 0 || d >= nz) continue;
                            if (keys[IDX(a, b, d)] < kp) { best = 0; break; }
                        }
                    }
                }
                sel[p] = (uint8_t)best;
                nsel += best;
            }
    return nsel;
}

/* Total of the interface-dependent energy of Eq. (4flip):
 * c_N sum chi (S - W) + h^3 sum_{solvent} U.  Used by the exactness checks. */
static double energy_now(int nx, int ny, int nz, const uint8_t *chi,
                         const double *U, int r, const int *qw, const int64_t *k3,
                         double cN, int64_t S, double h3, int64_t *Wtmp)
{
    int64_t G = (int64_t)nx * ny * nz;
    conv_any(nx, ny, nz, chi, r, qw, k3, Wtmp);
    int64_t s = or_surface_sum(G, chi, Wtmp, S);
    double v = 0.0;
    for (int64_t p = 0; p < G; ++p)
        if (!chi[p]) v += U[p];
    return cN * (double)s + h3 * v;
}

double or_energy(int nx, int ny, int nz, const uint8_t *chi, const double *U,
                 int r, const int *qw, const int64_t *k3, double cN, int64_t S,
                 double h3)
{
    int64_t G = (int64_t)nx * ny * nz;
    int64_t *W = (int64_t *)malloc(sizeof(int64_t) * G);
    double e = energy_now(nx, ny, nz, chi, U, r, qw, k3, cN, S, h3, W);
    free(W);
    return e;
}

/* Rounds of the parallel rule until no candidate has dE < 0.
 * Returns the number of rounds that flipped cells; round_flips (optional,
 * length max_rounds) records the flips of each round.  With verify != 0 the
 * energy is recomputed from scratch around every round and the largest
 * |(E_after - E_before) - sum dE| is returned in *verify_err. */
int or_blsm_parallel(int nx, int ny, int nz, uint8_t *chi, const double *U,
                     int r, const int *qw, const int64_t *k3, double cN, int64_t S,
                     int64_t k0, double h3, int max_rounds, int64_t *flips_out,
                     double *dEsum_out, int64_t *round_flips, int verify,
                     double *verify_err)
{
    int64_t G = (int64_t)nx * ny * nz;
    int64_t *W = (int64_t *)malloc(sizeof(int64_t) * G);
    int64_t *Wt = verify ? (int64_t *)malloc(sizeof(int64_t) * G) : NULL;
    double *dE = (double *)malloc(sizeof(double) * G);
    uint8_t *cand = (uint8_t *)malloc(G);
    uint8_t *sel = (uint8_t *)malloc(G);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * G);
    int rounds = 0;
    int64_t flips = 0;
    double dsum = 0.0, verr = 0.0;
    while (rounds < max_rounds) {
        conv_any(nx, ny, nz, chi, r, qw, k3, W);
        or_delta_e(nx, ny, nz, chi, W, U, cN, S, k0, h3, dE, cand);
        int64_t n = or_select(nx, ny, nz, cand, dE, r, sel, keys);
        if (n == 0) break;
        double e0 = verify ? energy_now(nx, ny, nz, chi, U, r, qw, k3, cN, S, h3, Wt) : 0.0;
        double rs = 0.0;
        for (int64_t p = 0; p < G; ++p)
            if (sel[p]) {
                chi[p] ^= 1;
                rs += dE[p];
            }
        if (verify) {
            double e1 = energy_now(nx, ny, nz, chi, U, r, qw, k3, cN, S, h3, Wt);
            double err = fabs((e1 - e0) - rs);
            if (err > verr) verr = err;
        }
        if (round_flips) round_flips[rounds] = n;
        dsum += rs;
        flips += n;
        ++rounds;
    }
    *flips_out = flips;
    *dEsum_out = dsum;
    if (verify_err) *verify_err = verr;
    free(W); free(Wt); free(dE); free(cand); free(sel); free(keys);
    return rounds;
}

/* ------------------------------------------------------ serial min-heap
 * The paper's literal flipping process (Sec. 3.1, Steps 2.1-2.2): keep the
 * candidates' dE in a min-heap, flip the smallest while it is negative,
 * then update w and dE in the kernel window of the flipped cell and the
 * candidate set.  Ties go to the smaller linear index.  Stale heap entries
 * are skipped by a per-cell version stamp.
 */
typedef struct { double e; int64_t p; uint32_t v; } hent;

static int hless(const hent *a, const hent *b)
{
    return a->e < b->e || (a->e == b->e && a->p < b->p);
}

static void hpush(hent *h, int64_t *n, hent x)
{
    int64_t i = (*n)++;
    h[i] = x;
    while (i > 0) {
        int64_t par = (i - 1) / 2;
        if (!hless(&h[i], &h[par])) break;
        hent t = h[i]; h[i] = h[par]; h[par] = t;
        i = par;
    }
}

static hent hpop(hent *h, int64_t *n)
{
    hent top = h[0];
    h[0] = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, rr = l + 1, m = i;
        if (l < *n && hless(&h[l], &h[m])) m = l;
        if (rr < *n && hless(&h[rr], &h[m])) m = rr;
        if (m == i) break;
        hent t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

int64_t or_blsm_heap(int nx, int ny, int nz, uint8_t *chi, const double *U,
                     int r, const int *qw, const int64_t *k3, double cN, int64_t S,
                     int64_t k0, double h3, int64_t max_flips, double *dEsum_out,
                     int verify, double *verify_err)
{
    int64_t G = (int64_t)nx * ny * nz;
    const int wd = 2 * r + 1;
    int64_t *W = (int64_t *)malloc(sizeof(int64_t) * G);
    int64_t *Wt = verify ? (int64_t *)malloc(sizeof(int64_t) * G) : NULL;
    uint32_t *ver = (uint32_t *)calloc(G, sizeof(uint32_t));
    int64_t cap = 4 * G + 1024, hn = 0;
    hent *heap = (hent *)malloc(sizeof(hent) * cap);
    conv_any(nx, ny, nz, chi, r, qw, k3, W);
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                int64_t p = IDX(i, j, k);
                if (!is_candidate(nx, ny, nz, chi, i, j, k)) continue;
                double e = flip_energy(chi[p], W[p], U[p], cN, S, k0, h3);
                if (e < 0.0) hpush(heap, &hn, (hent){e, p, ver[p]});
            }
    int64_t flips = 0;
    double dsum = 0.0, verr = 0.0;
    double ecur = verify ? energy_now(nx, ny, nz, chi, U, r, qw, k3, cN, S, h3, Wt) : 0.0;
    while (hn > 0 && flips < max_flips) {
        hent t = hpop(heap, &hn);
        if (t.v != ver[t.p]) continue;          /* stale entry */
        int64_t p = t.p;
        int i = (int)(p / ((int64_t)ny * nz));
        int j = (int)((p / nz) % ny);
        int k = (int)(p % nz);
        int sgn = chi[p] ? -1 : 1;              /* +1: solvent -> solute */
        chi[p] ^= 1;
        ++flips;
        dsum += t.e;
        for (int a = -r; a <= r; ++a)
            for (int b = -r; b <= r; ++b)
                for (int d = -r; d <= r; ++d) {
                    int ii = i + a, jj = j + b, kk = k + d;
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
                    const int64_t kw = k3 ? k3[((a + r) * wd + (b + r)) * wd + (d + r)]
                                          : (int64_t)qw[a + r] * qw[b + r] * qw[d + r];
                    W[IDX(ii, jj, kk)] += sgn * kw;
                }
        for (int a = -r; a <= r; ++a)
            for (int b = -r; b <= r; ++b)
                for (int d = -r; d <= r; ++d) {
                    int ii = i + a, jj = j + b, kk = k + d;
                    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz) continue;
                    int64_t q = IDX(ii, jj, kk);
                    ver[q]++;
                    if (!is_candidate(nx, ny, nz, chi, ii, jj, kk)) continue;
                    double e = flip_energy(chi[q], W[q], U[q], cN, S, k0, h3);
                    if (e < 0.0) {
                        if (hn >= cap) {
                            cap *= 2;
                            heap = (hent *)realloc(heap, sizeof(hent) * cap);
                        }
                        hpush(heap, &hn, (hent){e, q, ver[q]});
                    }
                }
        if (verify) {
            double e1 = energy_now(nx, ny, nz, chi, U, r, qw, k3, cN, S, h3, Wt);
            double err = fabs((e1 - ecur) - t.e);
            if (err > verr) verr = err;
            ecur = e1;
        }
    }
    *dEsum_out = dsum;
    if (verify_err) *verify_err = verr;
    free(W); free(Wt); free(ver); free(heap);
    return flips;
}

/* Tight initial surface (Sec. 3.1, "Initial surfaces"): a cell is solute
 * when phi(x) = min_i (|x - r_i| - d_i) < 0 at its centre. */
void or_init_tight(int nx, int ny, int nz, double h, const double *origin,
                   int na, const double *xyz, const double *d, uint8_t *chi)
{
#pragma omp parallel for collapse(2)
    for (int i = 0; i < nx; ++i)
        for (int j = 0; j < ny; ++j)
            for (int k = 0; k < nz; ++k) {
                double x = origin[0] + (i + 0.5) * h;
                double y = origin[1] + (j + 0.5) * h;
                double z = origin[2] + (k + 0.5) * h;
                double phi = INFINITY;
                for (int a = 0; a < na; ++a) {
                    double dx = x - xyz[3 * a], dy = y - xyz[3 * a + 1], dz = z - xyz[3 * a + 2];
                    double v = sqrt(dx * dx + dy * dy + dz * dz) - d[a];
                    if (v < phi) phi = v;
                }
                chi[IDX(i, j, k)] = phi < 0.0;
            }
}

/* Same test at a list of cells (for sampled checks on large grids). */
void or_init_tight_at(int64_t np, const int64_t *cells, int nx, int ny, int nz,
                      double h, const double *origin, int na,
                      const double *xyz, const double *d, uint8_t *chi,
                      double *phi_out)
{
#pragma omp parallel for
    for (int64_t t = 0; t < np; ++t) {
        int64_t p = cells[t];
        int i = (int)(p / ((int64_t)ny * nz)), j = (int)((p / nz) % ny), k = (int)(p % nz);
        double x = origin[0] + (i + 0.5) * h;
        double y = origin[1] + (j + 0.5) * h;
        double z = origin[2] + (k + 0.5) * h;
        double phi = INFINITY;
        for (int a = 0; a < na; ++a) {
            double dx = x - xyz[3 * a], dy = y - xyz[3 * a + 1], dz = z - xyz[3 * a + 2];
            double v = sqrt(dx * dx + dy * dy + dz * dz) - d[a];
            if (v < phi) phi = v;
        }
        chi[t] = phi < 0.0;
        phi_out[t] = phi;
    }
}
