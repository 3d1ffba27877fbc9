/*
 * oracle.c -- plain, slow, serial FP64 reference of the D3Q19 BGK lattice-Boltzmann
 * time step on sparse geometries (Tomczak & Szafran, "A new GPU implementation for
 * lattice-Boltzmann simulations on sparse geometries").
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load this file's library. The CUDA library neither links, loads
 * nor shares any code, header or table with it.
 *
 * What it computes. Tiling changes only how nodes are addressed, so the method's
 * result is the plain dense lattice-Boltzmann update; this file writes that update
 * out on a dense flagged array, loop z -> y -> x -> i, in plain FP64, compiled with
 * -O2 -ffp-contract=off so that the same source gives the same bits on x86-64 and
 * aarch64 hosts.
 *
 *   Lattice   D3Q19, weights 1/3, 1/18 (x6), 1/36 (x12), c_s^2 = 1/3 (Sec. 2.2).
 *   Collision LBGK, Eq. 2, with the quasi-compressible equilibrium of Eq. 3 and the
 *             velocity of Eq. 5; discrete update Eq. 7.
 *   Streaming pull form, fused with collision (Sec. 2.3): every non-solid node
 *             gathers f_i from x - c_i; propagation only takes place between
 *             non-solid nodes (Sec. 3.4, Algorithm 2), otherwise halfway bounce-back
 *             (Sec. 2.2, walls: "velocity 0 and bounce-back").
 *   Tiling    Algorithm 1 (Sec. 3.1), uniform a^3 tiles from node (0,0,0), padding
 *             nodes solid, all-solid tiles dropped, tiles kept in discovery order.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   R1 direction numbering: 0 rest; 1 E(+x) 2 N(+y) 3 W(-x) 4 S(-y) 5 T(+z) 6 B(-z);
 *      7 NE 8 NW 9 SW 10 SE; 11 ET 12 EB 13 WT 14 WB; 15 NT 16 NB 17 ST 18 SB.
 *      Only e_3 = W = (-1,0,0) survives in the paper's Fig. 1 caption; it is kept.
 *   R2 body force: Guo et al. (2002) forcing, F a force density; u = (sum c f + F/2)/rho;
 *      source S_i = (1 - 1/(2 tau)) w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)].
 *   R3 walls: halfway bounce-back in pull form, f_i(x) <- A_opp(i)(x) when x - c_i is
 *      solid, lies in an all-solid tile, or lies outside the box on a non-periodic axis.
 *   R4 inlet: f*_i = f^eq_i(rho, u_in) with rho from the gathered f; outlet:
 *      f*_i = f^eq_i(rho_out, u) with u the local velocity (constant pressure,
 *      zero-gradient velocity). Stored values are post-collision populations f*.
 *   R5 periodic axes wrap node coordinates; the tile grid wraps with them.
 *   R6 reported velocity: u = (sum c f* - F/2)/rho from the stored post-collision f*.
 *   R7 tile index t = tx + Tx (ty + Ty tz); nonEmptyTiles holds t (a 4-byte packing of
 *      the tile corner, Sec. 3.3); tileMap[t] holds the tile's rank or -1.
 *
 * Dense layout used throughout: node n = x + nx (y + ny z); populations f[i*N + n].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

enum { SOLID = 0, FLUID = 1, INLET = 2, OUTLET = 3 };

/* D3Q19 velocities (reading R1) and weights (Sec. 2.2). */
static const int C[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0},
    {1, 0, 1}, {1, 0, -1}, {-1, 0, 1}, {-1, 0, -1},
    {0, 1, 1}, {0, 1, -1}, {0, -1, 1}, {0, -1, -1}};
static const double W[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* opposite direction: c_opp(i) = -c_i, found by search rather than tabulated */
static int opp(int i) {
    for (int k = 0; k < Q; k++)
        if (C[k][0] == -C[i][0] && C[k][1] == -C[i][1] && C[k][2] == -C[i][2]) return k;
    return -1;
}

int oracle_version(void) { return 1; }

/* Export the lattice tables so tests can check them against the paper's constants. */
void oracle_lattice(int32_t* c, double* w, int32_t* op) {
    for (int i = 0; i < Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = C[i][a];
        w[i] = W[i];
        op[i] = opp(i);
    }
}

/* ---------------------------------------------------------------------------- */
/* Equilibrium, Eq. 3 (quasi-compressible), c_s^2 = 1/3 so 1/c_s^2 = 3,
 * 1/(2 c_s^4) = 4.5 and 1/(2 c_s^2) = 1.5. */
static double feq(int i, double rho, const double u[3]) {
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Guo forcing source term (reading R2). */
static double guo(int i, double tau, const double u[3], const double F[3]) {
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    double cF = C[i][0] * F[0] + C[i][1] * F[1] + C[i][2] * F[2];
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    return (1.0 - 0.5 / tau) * W[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
}

/* Density and momentum sum of a set of 19 populations (Eq. 5 numerator). */
static void moments(const double f[Q], double* rho, double j[3]) {
    double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; i++) {
        r += f[i];
        jx += C[i][0] * f[i];
        jy += C[i][1] * f[i];
        jz += C[i][2] * f[i];
    }
    *rho = r;
    j[0] = jx;
    j[1] = jy;
    j[2] = jz;
}

/* Collision at one node (Eq. 7 right-hand side plus forcing and boundary closures).
 * f: populations gathered by streaming; out: post-collision populations. */
void oracle_collide(const double f[Q], int type, double tau, const double F[3],
                    const double u_in[3], double rho_out, double out[Q]) {
    double rho, j[3], u[3];
    moments(f, &rho, j);
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F[a]) / rho;
    if (type == INLET) {
        for (int i = 0; i < Q; i++) out[i] = feq(i, rho, u_in);
    } else if (type == OUTLET) {
        for (int i = 0; i < Q; i++) out[i] = feq(i, rho_out, u);
    } else {
        for (int i = 0; i < Q; i++) out[i] = f[i] - (f[i] - feq(i, rho, u)) / tau + guo(i, tau, u, F);
    }
}

/* ---------------------------------------------------------------------------- */
/* Collision models beyond quasi-compressible LBGK (the paper's other variants).
 *
 * eq = 0: quasi-compressible equilibrium, Eq. 3 with u from Eq. 5 (the default above).
 * eq = 1: incompressible equilibrium, Eq. 4 with u from Eq. 6: f^eq_i = w_i (rho +
 *         3 c.u + 4.5 (c.u)^2 - 1.5 u.u), u = sum c f (+ F/2 with Guo forcing, the
 *         reference density rho_0 = 1 taking the place of rho in u).
 * coll = 0: LBGK, Eq. 2 / Eq. 7.
 * coll = 1: multiple relaxation times, Eq. 8, in the D3Q19 moment basis of d'Humieres,
 *         Ginzburg, Krafczyk, Lallemand and Luo (Phil. Trans. R. Soc. A 360, 2002):
 *         m = M f, m* = m - S (m - m^eq) + (I - S/2) M G, f* = M^-1 m*, with
 *         m^eq = M f^eq (the projection of the equilibrium above, so that S = I/tau is
 *         LBGK exactly) and G_i = w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)] the Guo force
 *         term without its (1 - 1/(2 tau)) factor (Guo et al. 2002, in moment space).
 * rates: the 19 diagonal entries of S in moment order (below).
 *
 * Moment basis: each row is a polynomial in the velocity c (|c|^2 = c.c), evaluated
 * on the 19 velocities, in this order:
 *   0 rho = 1,                  1 e = 19 |c|^2 - 30,
 *   2 eps = (21 |c|^4 - 53 |c|^2 + 24) / 2,
 *   3 j_x = c_x,  4 q_x = (5 |c|^2 - 9) c_x,  5 j_y,  6 q_y,  7 j_z,  8 q_z,
 *   9 3p_xx = 3 c_x^2 - |c|^2,  10 3pi_xx = (3 |c|^2 - 5)(3 c_x^2 - |c|^2),
 *  11 p_ww = c_y^2 - c_z^2,     12 pi_ww = (3 |c|^2 - 5)(c_y^2 - c_z^2),
 *  13 p_xy = c_x c_y,  14 p_yz = c_y c_z,  15 p_xz = c_x c_z,
 *  16 m_x = (c_y^2 - c_z^2) c_x,  17 m_y = (c_z^2 - c_x^2) c_y,  18 m_z = (c_x^2 - c_y^2) c_z.
 * The rows are mutually orthogonal, so M^-1 = M^T diag(1 / |row|^2). */
static double basis(int k, const int c[3]) {
    const double x = c[0], y = c[1], z = c[2], cc = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1.0;
        case 1: return 19.0 * cc - 30.0;
        case 2: return (21.0 * cc * cc - 53.0 * cc + 24.0) / 2.0;
        case 3: return x;
        case 4: return (5.0 * cc - 9.0) * x;
        case 5: return y;
        case 6: return (5.0 * cc - 9.0) * y;
        case 7: return z;
        case 8: return (5.0 * cc - 9.0) * z;
        case 9: return 3.0 * x * x - cc;
        case 10: return (3.0 * cc - 5.0) * (3.0 * x * x - cc);
        case 11: return y * y - z * z;
        case 12: return (3.0 * cc - 5.0) * (y * y - z * z);
        case 13: return x * y;
        case 14: return y * z;
        case 15: return x * z;
        case 16: return (y * y - z * z) * x;
        case 17: return (z * z - x * x) * y;
        default: return (x * x - y * y) * z;
    }
}

/* The moment matrix M[k][i] (row-major), exported for the tests. */
void oracle_mrt_matrix(double* M) {
    for (int k = 0; k < Q; k++)
        for (int i = 0; i < Q; i++) M[k * Q + i] = basis(k, C[i]);
}

/* Equilibrium of either model (eq = 0 Eq. 3, eq = 1 Eq. 4). */
static double feq_m(int i, int eq, double rho, const double u[3]) {
    if (eq == 0) return feq(i, rho, u);
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[i] * (rho + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* Velocity used in the collision: Eq. 5 (eq = 0) or Eq. 6 (eq = 1), with F/2. */
static void velocity_m(int eq, double rho, const double j[3], const double F[3], double u[3]) {
    for (int a = 0; a < 3; a++) u[a] = eq == 0 ? (j[a] + 0.5 * F[a]) / rho : j[a] + 0.5 * F[a];
}

void oracle_collide_m(const double f[Q], int type, double tau, const double F[3], const double u_in[3],
                      double rho_out, int eq, int coll, const double rates[Q], double out[Q]) {
    if (eq == 0 && coll == 0) {
        oracle_collide(f, type, tau, F, u_in, rho_out, out);
        return;
    }
    double rho, j[3], u[3];
    moments(f, &rho, j);
    velocity_m(eq, rho, j, F, u);
    if (type == INLET) {
        for (int i = 0; i < Q; i++) out[i] = feq_m(i, eq, rho, u_in);
        return;
    }
    if (type == OUTLET) {
        for (int i = 0; i < Q; i++) out[i] = feq_m(i, eq, rho_out, u);
        return;
    }
    double fe[Q], G[Q];
    for (int i = 0; i < Q; i++) {
        double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
        double cF = C[i][0] * F[0] + C[i][1] * F[1] + C[i][2] * F[2];
        double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        fe[i] = feq_m(i, eq, rho, u);
        G[i] = W[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
    }
    if (coll == 0) {
        for (int i = 0; i < Q; i++) out[i] = f[i] - (f[i] - fe[i]) / tau + (1.0 - 0.5 / tau) * G[i];
        return;
    }
    /* MRT: relax in moment space, then back with M^-1 = M^T diag(1/|row|^2) */
    double M[Q][Q], mstar[Q];
    for (int k = 0; k < Q; k++)
        for (int i = 0; i < Q; i++) M[k][i] = basis(k, C[i]);
    for (int k = 0; k < Q; k++) {
        double m = 0.0, meq = 0.0, mG = 0.0, norm = 0.0;
        for (int i = 0; i < Q; i++) {
            m += M[k][i] * f[i];
            meq += M[k][i] * fe[i];
            mG += M[k][i] * G[i];
            norm += M[k][i] * M[k][i];
        }
        mstar[k] = (m - rates[k] * (m - meq) + (1.0 - 0.5 * rates[k]) * mG) / norm;
    }
    for (int i = 0; i < Q; i++) {
        double v = 0.0;
        for (int k = 0; k < Q; k++) v += M[k][i] * mstar[k];
        out[i] = v;
    }
}

/* Zou-He boundary (Zou & He, Phys. Fluids 9, 1997; the D3Q19 form with the transverse
 * momentum correction of Hecht & Harting, J. Stat. Mech. 2010) at a node on box face
 * `face` (0: x = 0, 1: x = nx - 1, 2: y = 0, ..., 5: z = nz - 1), whose inward normal is
 * n = +e_a on the low faces and -e_a on the high ones (a = face / 2). The populations with
 * c.n > 0 come from outside and are unknown; with B = sum_{c.n=0} f + 2 sum_{c.n<0} f:
 *   velocity (kind 0, u_b given):  rho = B / (1 - u_b.n), j = rho u_b (eq 0);
 *                                  j = u_b, rho = B + u_b.n (eq 1, Eq. 6);
 *   pressure (kind 1, rho_b given, tangential velocity 0): rho = rho_b,
 *                                  j = rho_b (1 - B / rho_b) n (eq 0); j = (rho_b - B) n (eq 1);
 * then, j_n = j.n, for the unknown along n:    f_i = f_opp(i) + j_n / 3,
 * and for each unknown c_i = n + t e_b (t = +-1, b the tangential axis):
 *   f_i = f_opp(i) + (j_n + t j_b) / 6 - t N_b,  N_b = 1/2 sum_{c.n=0} c_b f - j_b / 3,
 * which makes the node's density rho and momentum j exactly. out: the completed set. */
void oracle_zou_he(const double f[Q], int face, int kind, int eq, const double u_b[3], double rho_b,
                   double out[Q]) {
    const int a = face / 2;
    const int sg = (face % 2 == 0) ? 1 : -1;
    double B = 0.0, T[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) {
        const int cn = C[i][a] * sg;
        if (cn == 0) {
            B += f[i];
            for (int b = 0; b < 3; b++) T[b] += C[i][b] * f[i];
        } else if (cn < 0) {
            B += 2.0 * f[i];
        }
    }
    double rho, j[3];
    if (kind == 0) {
        const double un = u_b[a] * sg;
        rho = eq == 0 ? B / (1.0 - un) : B + un;
        for (int b = 0; b < 3; b++) j[b] = eq == 0 ? rho * u_b[b] : u_b[b];
    } else {
        rho = rho_b;
        const double jn = eq == 0 ? rho_b * (1.0 - B / rho_b) : rho_b - B;
        for (int b = 0; b < 3; b++) j[b] = 0.0;
        j[a] = jn * sg;
    }
    const double jn = j[a] * sg;
    for (int i = 0; i < Q; i++) out[i] = f[i];
    for (int i = 0; i < Q; i++) {
        if (C[i][a] * sg <= 0) continue;
        double v = f[opp(i)];
        int tang = -1;
        for (int b = 0; b < 3; b++)
            if (b != a && C[i][b] != 0) tang = b;
        if (tang < 0) {
            v += jn / 3.0;
        } else {
            const int t = C[i][tang];
            const double N = 0.5 * T[tang] - j[tang] / 3.0;
            v += (jn + t * j[tang]) / 6.0 - t * N;
        }
        out[i] = v;
    }
    (void)rho;
}

/* oracle_step with a collision model (eq, coll, rates as for oracle_collide_m) and an
 * optional moving wall: lid_face 0..5 = the box face x = -1, x = nx, y = -1, y = ny,
 * z = -1, z = nz (a non-periodic axis), or -1 for none. A link whose source x - c_i lies
 * beyond that face bounces back from a wall moving with velocity lid_u (Ladd 1994, the
 * wall density taken as the reference density 1):
 *     f_i(x) = f*_opp(i)(x) + 6 w_i (c_i . lid_u). */
void oracle_step_m(const double* A, double* B, const uint8_t* nt, int nx, int ny, int nz, unsigned periodic,
                   double tau, const double g[3], const double* g_field, const double u_in[3], double rho_out,
                   int eq, int coll, const double rates[Q], int lid_face, const double lid_u[3], int bc,
                   int in_face, int out_face, int nthreads);

/* Macroscopic fields of either model: u = (sum c f* - F/2) / rho (eq = 0, reading R6) or
 * u = sum c f* - F/2 (eq = 1, Eq. 6). */
void oracle_macroscopic_m(const double* f, const uint8_t* nt, long N, const double g[3], const double* g_field,
                          int eq, double* rho, double* u);

/* ---------------------------------------------------------------------------- */
/* Streaming source of direction i at node (x,y,z): the node x - c_i, wrapped on
 * periodic axes (bit 0: x, bit 1: y, bit 2: z). Returns 0 when it leaves the box. */
static int source_node(int x, int y, int z, int i, int nx, int ny, int nz,
                       unsigned periodic, long* src) {
    int p[3] = {x - C[i][0], y - C[i][1], z - C[i][2]};
    int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++) {
        if (p[a] < 0 || p[a] >= n[a]) {
            if (!(periodic & (1u << a))) return 0;
            p[a] = (p[a] + n[a]) % n[a];
        }
    }
    *src = p[0] + (long)nx * (p[1] + (long)ny * p[2]);
    return 1;
}

static void force_at(long n, const double g[3], const double* g_field, double F[3]) {
    F[0] = g_field ? g_field[n] : g[0];
    F[1] = g[1];
    F[2] = g[2];
}

/* One fused pull step A -> B on the dense array (Algorithm 2 without tiles).
 * g_field, when not NULL, is the per-node x body force replacing g[0].
 * Solid nodes of B are left untouched. */
void oracle_step(const double* A, double* B, const uint8_t* nt, int nx, int ny, int nz,
                 unsigned periodic, double tau, const double g[3], const double* g_field,
                 const double u_in[3], double rho_out, int nthreads) {
    long N = (long)nx * ny * nz;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long n = x + (long)nx * (y + (long)ny * z);
                if (nt[n] == SOLID) continue;
                double f[Q], out[Q], F[3];
                for (int i = 0; i < Q; i++) {
                    long s;
                    if (source_node(x, y, z, i, nx, ny, nz, periodic, &s) && nt[s] != SOLID)
                        f[i] = A[i * N + s];
                    else
                        f[i] = A[opp(i) * N + n];
                }
                force_at(n, g, g_field, F);
                oracle_collide(f, nt[n], tau, F, u_in, rho_out, out);
                for (int i = 0; i < Q; i++) B[i * N + n] = out[i];
            }
}

/* Does the link of direction i at node (x,y,z) come from beyond box face `face`? */
static int beyond_face(int x, int y, int z, int i, int nx, int ny, int nz, int face) {
    if (face < 0) return 0;
    const int a = face / 2;
    const int q = (a == 0 ? x : a == 1 ? y : z) - C[i][a];
    const int n = a == 0 ? nx : a == 1 ? ny : nz;
    return (face % 2 == 0) ? q < 0 : q >= n;
}

void oracle_step_m(const double* A, double* B, const uint8_t* nt, int nx, int ny, int nz, unsigned periodic,
                   double tau, const double g[3], const double* g_field, const double u_in[3], double rho_out,
                   int eq, int coll, const double rates[Q], int lid_face, const double lid_u[3], int bc,
                   int in_face, int out_face, int nthreads) {
    long N = (long)nx * ny * nz;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long n = x + (long)nx * (y + (long)ny * z);
                if (nt[n] == SOLID) continue;
                double f[Q], out[Q], F[3];
                for (int i = 0; i < Q; i++) {
                    long s;
                    if (source_node(x, y, z, i, nx, ny, nz, periodic, &s) && nt[s] != SOLID) {
                        f[i] = A[i * N + s];
                    } else {
                        f[i] = A[opp(i) * N + n];
                        if (beyond_face(x, y, z, i, nx, ny, nz, lid_face))
                            f[i] += 6.0 * W[i] * (C[i][0] * lid_u[0] + C[i][1] * lid_u[1] + C[i][2] * lid_u[2]);
                    }
                }
                force_at(n, g, g_field, F);
                if (bc == 1 && (nt[n] == INLET || nt[n] == OUTLET)) {
                    /* Zou-He: complete the unknown populations, then collide as fluid */
                    double fz[Q];
                    if (nt[n] == INLET) oracle_zou_he(f, in_face, 0, eq, u_in, 1.0, fz);
                    else oracle_zou_he(f, out_face, 1, eq, u_in, rho_out, fz);
                    oracle_collide_m(fz, FLUID, tau, F, u_in, rho_out, eq, coll, rates, out);
                } else {
                    oracle_collide_m(f, nt[n], tau, F, u_in, rho_out, eq, coll, rates, out);
                }
                for (int i = 0; i < Q; i++) B[i * N + n] = out[i];
            }
}

/* Equilibrium initial state f = f^eq(rho0, u0) at non-solid nodes, NaN at solid. */
void oracle_init(double* f, const uint8_t* nt, long N, double rho0, const double u0[3]) {
    for (long n = 0; n < N; n++)
        for (int i = 0; i < Q; i++) f[i * N + n] = nt[n] == SOLID ? NAN : feq(i, rho0, u0);
}

/* Macroscopic fields from stored post-collision populations (reading R6):
 * rho = sum f*, u = (sum c f* - F/2)/rho; zero at solid nodes. u is [3][N]. */
void oracle_macroscopic(const double* f, const uint8_t* nt, long N, const double g[3],
                        const double* g_field, double* rho, double* u) {
    for (long n = 0; n < N; n++) {
        if (nt[n] == SOLID) {
            rho[n] = 0.0;
            u[n] = u[N + n] = u[2 * N + n] = 0.0;
            continue;
        }
        double fl[Q], r, j[3], F[3];
        for (int i = 0; i < Q; i++) fl[i] = f[i * N + n];
        moments(fl, &r, j);
        force_at(n, g, g_field, F);
        rho[n] = r;
        for (int a = 0; a < 3; a++) u[a * N + n] = (j[a] - 0.5 * F[a]) / r;
    }
}

void oracle_macroscopic_m(const double* f, const uint8_t* nt, long N, const double g[3], const double* g_field,
                          int eq, double* rho, double* u) {
    if (eq == 0) {
        oracle_macroscopic(f, nt, N, g, g_field, rho, u);
        return;
    }
    for (long n = 0; n < N; n++) {
        if (nt[n] == SOLID) {
            rho[n] = 0.0;
            u[n] = u[N + n] = u[2 * N + n] = 0.0;
            continue;
        }
        double fl[Q], r, j[3], F[3];
        for (int i = 0; i < Q; i++) fl[i] = f[i * N + n];
        moments(fl, &r, j);
        force_at(n, g, g_field, F);
        rho[n] = r;
        for (int a = 0; a < 3; a++) u[a * N + n] = j[a] - 0.5 * F[a];
    }
}

/* Global mass and momentum over non-solid nodes: out = {sum f*, sum (sum c f* - F/2)}. */
void oracle_reduce(const double* f, const uint8_t* nt, long N, const double g[3],
                   const double* g_field, double out[4]) {
    double m = 0.0, p[3] = {0.0, 0.0, 0.0};
    for (long n = 0; n < N; n++) {
        if (nt[n] == SOLID) continue;
        double fl[Q], r, j[3], F[3];
        for (int i = 0; i < Q; i++) fl[i] = f[i * N + n];
        moments(fl, &r, j);
        force_at(n, g, g_field, F);
        m += r;
        for (int a = 0; a < 3; a++) p[a] += j[a] - 0.5 * F[a];
    }
    out[0] = m;
    out[1] = p[0];
    out[2] = p[1];
    out[3] = p[2];
}

/* ---------------------------------------------------------------------------- */
/* Algorithm 1 (Sec. 3.1): cover the geometry with a^3 tiles from node (0,0,0), padding
 * nodes being solid, and keep a tile as soon as one of its nodes is not solid.
 * tile_map has Tx*Ty*Tz entries (T = ceil(n/a)); returns the number of tiles kept. */
long oracle_tiling(const uint8_t* nt, int nx, int ny, int nz, int a, int32_t* tile_map,
                   uint32_t* non_empty) {
    int Tx = (nx + a - 1) / a, Ty = (ny + a - 1) / a, Tz = (nz + a - 1) / a;
    long count = 0;
    for (int tz = 0; tz < Tz; tz++)
        for (int ty = 0; ty < Ty; ty++)
            for (int tx = 0; tx < Tx; tx++) {
                long t = tx + (long)Tx * (ty + (long)Ty * tz);
                int keep = 0;
                for (int dz = 0; dz < a && !keep; dz++)
                    for (int dy = 0; dy < a && !keep; dy++)
                        for (int dx = 0; dx < a && !keep; dx++) {
                            int x = a * tx + dx, y = a * ty + dy, z = a * tz + dz;
                            if (x >= nx || y >= ny || z >= nz) continue; /* padding: solid */
                            if (nt[x + (long)nx * (y + (long)ny * z)] != SOLID) keep = 1;
                        }
                if (keep) {
                    tile_map[t] = (int32_t)count;
                    non_empty[count] = (uint32_t)t;
                    count++;
                } else {
                    tile_map[t] = -1;
                }
            }
    return count;
}

/* Dense <-> tile-major conversion for the tiled CPU stepper. Tile-major layout:
 * ft[(k*Q + i)*64 + s], s = xt + 4 yt + 16 zt (the XYZ order of Eq. 11), k the tile rank.
 * Padding slots hold NaN (values) or SOLID (types). */
static void tile_origin(uint32_t t, int Tx, int Ty, int* ox, int* oy, int* oz) {
    *ox = 4 * (int)(t % (uint32_t)Tx);
    *oy = 4 * (int)((t / (uint32_t)Tx) % (uint32_t)Ty);
    *oz = 4 * (int)(t / ((uint32_t)Tx * (uint32_t)Ty));
}

void oracle_to_tiles(const double* f, const uint8_t* nt, int nx, int ny, int nz,
                     const uint32_t* non_empty, long n_tiles, double* ft, uint8_t* ntt) {
    long N = (long)nx * ny * nz;
    int Tx = (nx + 3) / 4, Ty = (ny + 3) / 4;
    for (long k = 0; k < n_tiles; k++) {
        int ox, oy, oz;
        tile_origin(non_empty[k], Tx, Ty, &ox, &oy, &oz);
        for (int s = 0; s < 64; s++) {
            int x = ox + (s & 3), y = oy + ((s >> 2) & 3), z = oz + (s >> 4);
            int in = x < nx && y < ny && z < nz;
            long n = in ? x + (long)nx * (y + (long)ny * z) : 0;
            if (ntt) ntt[k * 64 + s] = in ? nt[n] : SOLID;
            if (f)
                for (int i = 0; i < Q; i++) ft[(k * Q + i) * 64 + s] = in ? f[i * N + n] : NAN;
        }
    }
}

void oracle_from_tiles(const double* ft, int nx, int ny, int nz, const uint32_t* non_empty,
                       long n_tiles, double* f) {
    long N = (long)nx * ny * nz;
    int Tx = (nx + 3) / 4, Ty = (ny + 3) / 4;
    for (long n = 0; n < (long)Q * N; n++) f[n] = NAN;
    for (long k = 0; k < n_tiles; k++) {
        int ox, oy, oz;
        tile_origin(non_empty[k], Tx, Ty, &ox, &oy, &oz);
        for (int s = 0; s < 64; s++) {
            int x = ox + (s & 3), y = oy + ((s >> 2) & 3), z = oz + (s >> 4);
            if (x >= nx || y >= ny || z >= nz) continue;
            long n = x + (long)nx * (y + (long)ny * z);
            for (int i = 0; i < Q; i++) f[i * N + n] = ft[(k * Q + i) * 64 + s];
        }
    }
}

/* Tiled CPU stepper: the same arithmetic as oracle_step, with nodes addressed through
 * tileMap / nonEmptyTiles (Sec. 3.1-3.2). A source in an all-solid tile is solid.
 * Periodic axes need dimensions divisible by 4. g_field, when given, is tile-major
 * [k*64 + s]. */
void oracle_step_tiled(const double* At, double* Bt, const uint8_t* ntt, const int32_t* tile_map,
                       const uint32_t* non_empty, long n_tiles, int nx, int ny, int nz,
                       unsigned periodic, double tau, const double g[3], const double* g_field,
                       const double u_in[3], double rho_out) {
    int Tx = (nx + 3) / 4, Ty = (ny + 3) / 4;
    for (long k = 0; k < n_tiles; k++) {
        int ox, oy, oz;
        tile_origin(non_empty[k], Tx, Ty, &ox, &oy, &oz);
        for (int s = 0; s < 64; s++) {
            if (ntt[k * 64 + s] == SOLID) continue;
            int x = ox + (s & 3), y = oy + ((s >> 2) & 3), z = oz + (s >> 4);
            double f[Q], out[Q], F[3];
            for (int i = 0; i < Q; i++) {
                long src_k = -1;
                int src_s = 0;
                long sn;
                if (source_node(x, y, z, i, nx, ny, nz, periodic, &sn)) {
                    int sx = (int)(sn % nx), sy = (int)((sn / nx) % ny), sz = (int)(sn / ((long)nx * ny));
                    long t = sx / 4 + (long)Tx * (sy / 4 + (long)Ty * (sz / 4));
                    src_k = tile_map[t];
                    src_s = (sx & 3) + 4 * (sy & 3) + 16 * (sz & 3);
                }
                if (src_k >= 0 && ntt[src_k * 64 + src_s] != SOLID)
                    f[i] = At[(src_k * Q + i) * 64 + src_s];
                else
                    f[i] = At[(k * Q + opp(i)) * 64 + s];
            }
            F[0] = g_field ? g_field[k * 64 + s] : g[0];
            F[1] = g[1];
            F[2] = g[2];
            oracle_collide(f, ntt[k * 64 + s], tau, F, u_in, rho_out, out);
            for (int i = 0; i < Q; i++) Bt[(k * Q + i) * 64 + s] = out[i];
        }
    }
}

/* ---------------------------------------------------------------------------- */
/* Tangent-linear model of the step (forward-mode differentiation with dual numbers).
 * A dual carries a value and its directional derivative. */
typedef struct {
    double v, d;
} dual;
static dual dn(double v, double d) {
    dual r = {v, d};
    return r;
}
static dual dadd(dual a, dual b) { return dn(a.v + b.v, a.d + b.d); }
static dual dsub(dual a, dual b) { return dn(a.v - b.v, a.d - b.d); }
static dual dmul(dual a, dual b) { return dn(a.v * b.v, a.d * b.v + a.v * b.d); }
static dual ddiv(dual a, dual b) { return dn(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static dual dk(double c) { return dn(c, 0.0); }

static dual feq_tl(int i, dual rho, const dual u[3]) {
    dual cu = dadd(dadd(dmul(dk(C[i][0]), u[0]), dmul(dk(C[i][1]), u[1])), dmul(dk(C[i][2]), u[2]));
    dual uu = dadd(dadd(dmul(u[0], u[0]), dmul(u[1], u[1])), dmul(u[2], u[2]));
    dual poly = dsub(dadd(dadd(dk(1.0), dmul(dk(3.0), cu)), dmul(dmul(dk(4.5), cu), cu)),
                     dmul(dk(1.5), uu));
    return dmul(dmul(dk(W[i]), rho), poly);
}

static dual guo_tl(int i, dual tau, const dual u[3], const dual F[3]) {
    dual cu = dadd(dadd(dmul(dk(C[i][0]), u[0]), dmul(dk(C[i][1]), u[1])), dmul(dk(C[i][2]), u[2]));
    dual cF = dadd(dadd(dmul(dk(C[i][0]), F[0]), dmul(dk(C[i][1]), F[1])), dmul(dk(C[i][2]), F[2]));
    dual uF = dadd(dadd(dmul(u[0], F[0]), dmul(u[1], F[1])), dmul(u[2], F[2]));
    dual beta = dsub(dk(1.0), ddiv(dk(0.5), tau));
    dual q = dadd(dmul(dk(3.0), dsub(cF, uF)), dmul(dmul(dk(9.0), cu), cF));
    return dmul(dmul(beta, dk(W[i])), q);
}

static void collide_tl(const dual f[Q], int type, dual tau, const dual F[3], const double u_in[3],
                       double rho_out, dual out[Q]) {
    dual rho = dk(0.0), j[3] = {dk(0.0), dk(0.0), dk(0.0)}, u[3];
    for (int i = 0; i < Q; i++) {
        rho = dadd(rho, f[i]);
        for (int a = 0; a < 3; a++) j[a] = dadd(j[a], dmul(dk(C[i][a]), f[i]));
    }
    for (int a = 0; a < 3; a++) u[a] = ddiv(dadd(j[a], dmul(dk(0.5), F[a])), rho);
    if (type == INLET) {
        dual uin[3] = {dk(u_in[0]), dk(u_in[1]), dk(u_in[2])};
        for (int i = 0; i < Q; i++) out[i] = feq_tl(i, rho, uin);
    } else if (type == OUTLET) {
        for (int i = 0; i < Q; i++) out[i] = feq_tl(i, dk(rho_out), u);
    } else {
        for (int i = 0; i < Q; i++)
            out[i] = dadd(dsub(f[i], ddiv(dsub(f[i], feq_tl(i, rho, u)), tau)), guo_tl(i, tau, u, F));
    }
}

/* Tangent step: (B, dB) = (step(A), J_A dA + J_tau dtau + J_g dg). dg_field is the
 * tangent of the per-node x force (dense) or NULL; dg is the tangent of uniform g. */
void oracle_step_tl(const double* A, const double* dA, double* B, double* dB, const uint8_t* nt,
                    int nx, int ny, int nz, unsigned periodic, double tau, double dtau,
                    const double g[3], const double dg[3], const double* g_field,
                    const double* dg_field, const double u_in[3], double rho_out) {
    long N = (long)nx * ny * nz;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long n = x + (long)nx * (y + (long)ny * z);
                if (nt[n] == SOLID) continue;
                dual f[Q], out[Q], F[3];
                for (int i = 0; i < Q; i++) {
                    long s;
                    if (source_node(x, y, z, i, nx, ny, nz, periodic, &s) && nt[s] != SOLID)
                        f[i] = dn(A[i * N + s], dA[i * N + s]);
                    else
                        f[i] = dn(A[opp(i) * N + n], dA[opp(i) * N + n]);
                }
                F[0] = dn(g_field ? g_field[n] : g[0], dg_field ? dg_field[n] : dg[0]);
                F[1] = dn(g[1], dg[1]);
                F[2] = dn(g[2], dg[2]);
                collide_tl(f, nt[n], dn(tau, dtau), F, u_in, rho_out, out);
                for (int i = 0; i < Q; i++) {
                    B[i * N + n] = out[i].v;
                    dB[i * N + n] = out[i].d;
                }
            }
}

/* ---------------------------------------------------------------------------- */
/* Reverse-mode adjoint of oracle_collide, derived by hand. lam: adjoint of the 19
 * outputs; mu: adjoint of the 19 gathered inputs (written); Fbar, taubar accumulate. */
void oracle_collide_adj(const double f[Q], int type, double tau, const double F[3],
                        const double u_in[3], double rho_out, const double lam[Q], double mu[Q],
                        double Fbar[3], double* taubar) {
    double rho, j[3], u[3];
    moments(f, &rho, j);
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * F[a]) / rho;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double rhobar = 0.0, ubar[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) mu[i] = 0.0;
    if (type == INLET) {
        for (int i = 0; i < Q; i++) {
            double cu = C[i][0] * u_in[0] + C[i][1] * u_in[1] + C[i][2] * u_in[2];
            double ui2 = u_in[0] * u_in[0] + u_in[1] * u_in[1] + u_in[2] * u_in[2];
            rhobar += lam[i] * W[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * ui2);
        }
        for (int i = 0; i < Q; i++) mu[i] = rhobar;
        return;
    }
    if (type == OUTLET) {
        for (int i = 0; i < Q; i++) {
            double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
            for (int a = 0; a < 3; a++)
                ubar[a] += lam[i] * W[i] * rho_out * (3.0 * C[i][a] + 9.0 * cu * C[i][a] - 3.0 * u[a]);
        }
    } else {
        double beta = 1.0 - 0.5 / tau;
        double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        double tb = 0.0;
        for (int i = 0; i < Q; i++) {
            double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
            double cF = C[i][0] * F[0] + C[i][1] * F[1] + C[i][2] * F[2];
            double e = 1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu;
            double fe = W[i] * rho * e;
            double qi = 3.0 * (cF - uF) + 9.0 * cu * cF;
            /* out_i = f_i - (f_i - fe_i)/tau + beta w_i q_i */
            mu[i] += lam[i] * (1.0 - 1.0 / tau);
            double feqbar = lam[i] / tau;
            tb += lam[i] * (f[i] - fe) / (tau * tau) + lam[i] * W[i] * qi * 0.5 / (tau * tau);
            rhobar += feqbar * W[i] * e;
            for (int a = 0; a < 3; a++) {
                ubar[a] += feqbar * W[i] * rho * (3.0 * C[i][a] + 9.0 * cu * C[i][a] - 3.0 * u[a]);
                ubar[a] += lam[i] * beta * W[i] * (-3.0 * F[a] + 9.0 * C[i][a] * cF);
                Fbar[a] += lam[i] * beta * W[i] * (3.0 * C[i][a] - 3.0 * u[a] + 9.0 * cu * C[i][a]);
            }
        }
        *taubar += tb;
    }
    /* u = (j + F/2) / rho */
    double jbar[3];
    for (int a = 0; a < 3; a++) {
        jbar[a] = ubar[a] / rho;
        Fbar[a] += 0.5 * ubar[a] / rho;
        rhobar -= ubar[a] * u[a] / rho;
    }
    for (int i = 0; i < Q; i++) mu[i] += rhobar + C[i][0] * jbar[0] + C[i][1] * jbar[1] + C[i][2] * jbar[2];
}

/* Adjoint of one step: given the state A = s_t and lam_next = dL/ds_{t+1}, writes
 * lam = dL/ds_t (the transpose of gather + collision, formed by scatter-adding), and
 * accumulates dL/dF: per node into gbar_field (x component, dense) when not NULL, and
 * summed into gbar[3]; dL/dtau into *taubar. */
void oracle_step_adj(const double* A, const double* lam_next, double* lam, const uint8_t* nt,
                     int nx, int ny, int nz, unsigned periodic, double tau, const double g[3],
                     const double* g_field, const double u_in[3], double rho_out,
                     double* gbar_field, double gbar[3], double* taubar) {
    long N = (long)nx * ny * nz;
    for (long n = 0; n < (long)Q * N; n++) lam[n] = 0.0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long n = x + (long)nx * (y + (long)ny * z);
                if (nt[n] == SOLID) continue;
                double f[Q], l[Q], mu[Q], F[3], Fb[3] = {0.0, 0.0, 0.0};
                long src[Q];
                for (int i = 0; i < Q; i++) {
                    long s;
                    if (source_node(x, y, z, i, nx, ny, nz, periodic, &s) && nt[s] != SOLID) {
                        src[i] = s;
                        f[i] = A[i * N + s];
                    } else {
                        src[i] = -1;
                        f[i] = A[opp(i) * N + n];
                    }
                    l[i] = lam_next[i * N + n];
                }
                force_at(n, g, g_field, F);
                oracle_collide_adj(f, nt[n], tau, F, u_in, rho_out, l, mu, Fb, taubar);
                for (int i = 0; i < Q; i++) {
                    if (src[i] >= 0)
                        lam[i * N + src[i]] += mu[i];
                    else
                        lam[opp(i) * N + n] += mu[i];
                }
                if (gbar_field) gbar_field[n] += Fb[0];
                for (int a = 0; a < 3; a++) gbar[a] += Fb[a];
            }
}

/* Outlet-flux loss L = mean over non-solid nodes of the plane x = plane_x of
 * u_x = (sum c_x f* - F_x/2)/rho. Writes lam = dL/df (zero off the plane) and adds the
 * direct dL/dF_x to gbar_field (dense, may be NULL) and gbar[0]. Returns L. */
double oracle_loss(const double* f, const uint8_t* nt, int nx, int ny, int nz, int plane_x,
                   const double g[3], const double* g_field, double* lam, double* gbar_field,
                   double gbar[3]) {
    long N = (long)nx * ny * nz;
    long count = 0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            if (nt[plane_x + (long)nx * (y + (long)ny * z)] != SOLID) count++;
    for (long n = 0; n < (long)Q * N; n++) lam[n] = 0.0;
    if (count == 0) return 0.0;
    double L = 0.0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++) {
            long n = plane_x + (long)nx * (y + (long)ny * z);
            if (nt[n] == SOLID) continue;
            double fl[Q], r, j[3], F[3];
            for (int i = 0; i < Q; i++) fl[i] = f[i * N + n];
            moments(fl, &r, j);
            force_at(n, g, g_field, F);
            double ux = (j[0] - 0.5 * F[0]) / r;
            L += ux;
            for (int i = 0; i < Q; i++) lam[i * N + n] = (C[i][0] - ux) / r / (double)count;
            double d = -0.5 / r / (double)count;
            if (gbar_field) gbar_field[n] += d;
            gbar[0] += d;
        }
    return L / (double)count;
}
