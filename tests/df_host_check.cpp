// Host build of the FP64 step's hybrid arithmetic (the double-float helpers and the LBGK +
// Guo collision that the CUDA kernel compiles from the same header), checked against
// long-double evaluations. Prints one "name value" line per measured quantity; the pytest
// wrapper (test_df_host.py) holds the bounds.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../paper_1611_02445_gb300/csrc/lbm_collide_df.cuh"

using namespace lbm;
typedef long double LD;

// D3Q19 velocities in the library's numbering: 0 rest; 1 E 2 N 3 W 4 S 5 T 6 B;
// 7 NE 8 NW 9 SW 10 SE; 11 ET 12 EB 13 WT 14 WB; 15 NT 16 NB 17 ST 18 SB.
static const int CV[19][3] = {{0, 0, 0},  {1, 0, 0},   {0, 1, 0},  {-1, 0, 0}, {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {1, 0, 1},  {1, 0, -1}, {-1, 0, 1},
                              {-1, 0, -1}, {0, 1, 1},  {0, 1, -1}, {0, -1, 1}, {0, -1, -1}};
static LD weight(int i) { return i == 0 ? 1.0L / 3 : (i < 7 ? 1.0L / 18 : 1.0L / 36); }

int main() {
    std::mt19937_64 rng(20240611);
    std::uniform_real_distribution<double> U(0.0, 1.0);

    // fix_from_double: d 2^58 rounded to nearest, ties away from zero (exact reference)
    long fix_bad = 0;
    for (int n = 0; n < 2000000; n++) {
        const double d = std::ldexp(1.0 + U(rng), -(int)(rng() % 24)) * ((rng() & 1) ? -1.0 : 1.0);
        const LD ref = roundl((LD)d * 0x1p58L);
        if ((LD)fix_from_double(d) != ref) fix_bad++;
    }
    std::printf("fix_mismatches %ld\n", fix_bad);

    // fix_from_double_cvt: d 2^58 rounded to nearest, ties to even, including ties
    long cvt_bad = 0;
    for (int n = 0; n < 2000000; n++) {
        double d = std::ldexp(1.0 + U(rng), -(int)(rng() % 30)) * ((rng() & 1) ? -1.0 : 1.0);
        if (n % 4 == 0) d = std::ldexp(std::floor(std::ldexp(d, 58)) + 0.5, -58);   // an exact tie
        const LD ref = nearbyintl((LD)d * 0x1p58L);                                     // ties to even
        if ((LD)fix_from_double_cvt(d) != ref) cvt_bad++;
    }
    if (fix_from_double_cvt(0.0) != 0 || fix_from_double_cvt(-0.0) != 0 || fix_from_double_cvt(1e-310) != 0) cvt_bad++;
    std::printf("fix_cvt_mismatches %ld\n", cvt_bad);

    // fix_from_double_fast: flags exactly the inputs outside [2^-6, 16) (negative, zero,
    // subnormal, infinite and NaN included) and agrees with fix_from_double on all others
    long fast_bad = 0, fast_flag = 0;
    for (int n = 0; n < 2000000; n++) {
        double d = std::ldexp(1.0 + U(rng), (int)(rng() % 16) - 10) * ((rng() % 8 == 0) ? -1.0 : 1.0);
        if (n % 1000 == 1) d = 0.0;
        if (n % 1000 == 2) d = -0.0;
        if (n % 1000 == 3) d = 1e-310;
        if (n % 1000 == 4) d = INFINITY;
        if (n % 1000 == 5) d = NAN;
        if (n % 1000 == 6) d = 0x1p-6;
        if (n % 1000 == 7) d = std::nextafter(0x1p-6, 0.0);
        if (n % 1000 == 8) d = std::nextafter(16.0, 0.0);
        if (n % 1000 == 9) d = 16.0;
        bool bad = false;
        const int64_t v = fix_from_double_fast(d, bad);
        const bool inside = d >= 0x1p-6 && d < 16.0;
        if (bad == inside) fast_flag++;
        if (!bad && v != fix_from_double(d)) fast_bad++;
    }
    std::printf("fix_fast_mismatches %ld\n", fast_bad);
    std::printf("fix_fast_flag_errors %ld\n", fast_flag);

    // df_from_fix: relative error of hi + lo against x 2^-58
    double fix_rel = 0;
    for (int n = 0; n < 2000000; n++) {
        const int sh = (int)(rng() % 63);
        int64_t x = (int64_t)(rng() >> (64 - sh - 1));
        if (rng() & 1) x = -x;
        if (x == 0) continue;
        const dfl p = df_from_fix(x);
        const LD ex = (LD)x * 0x1p-58L;
        fix_rel = std::fmax(fix_rel, (double)(fabsl((LD)p.h + (LD)p.l - ex) / fabsl(ex)));
    }
    std::printf("df_from_fix_rel %.3e\n", fix_rel);

    // df_from_double: relative error against d, 2^-40 <= |d| < 2
    double dbl_rel = 0;
    for (int n = 0; n < 2000000; n++) {
        const double d = std::ldexp(1.0 + U(rng), -(int)(rng() % 40)) * ((rng() & 1) ? -1.0 : 1.0);
        const dfl p = df_from_double(d);
        dbl_rel = std::fmax(dbl_rel, (double)(fabsl((LD)p.h + (LD)p.l - (LD)d) / fabsl((LD)d)));
    }
    std::printf("df_from_double_rel %.3e\n", dbl_rel);

    // df_to_double_pos: the nearest double to hi + lo (normalised positive pairs)
    long round_bad = 0;
    for (int n = 0; n < 2000000; n++) {
        const float h = (float)std::ldexp(1.0 + U(rng), -(int)(rng() % 30));
        const float l = (float)((U(rng) - 0.5) * std::ldexp((double)h, -24));
        const dfl p = df_make(h, l);
        const double ref = (double)((LD)h + (LD)l);   // exact sum, rounded once to nearest
        if (df_to_double_pos(p) != ref) round_bad++;
    }
    std::printf("to_double_mismatches %ld\n", round_bad);

    // collide_df against the LBGK + Guo update evaluated in long double
    double coll_abs = 0, mass_rel = 0;
    long fallback_states = 0;   // states with a population outside [2^-6, 16): the FP64-pipe moments
    for (int n = 0; n < 200000; n++) {
        const double tau = 0.51 + 1.5 * U(rng), omega = 1.0 / tau, beta = 1.0 - 0.5 / tau;
        const double F[3] = {1e-4 * (2 * U(rng) - 1), 1e-4 * (2 * U(rng) - 1), 1e-4 * (2 * U(rng) - 1)};
        const DFConst K = make_df_const(omega, beta, F[0], F[1], F[2]);
        double f[19];
        const double u0[3] = {0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1)};
        const double rho0 = 0.9 + 0.2 * U(rng);
        for (int i = 0; i < 19; i++) {
            const double cu = CV[i][0] * u0[0] + CV[i][1] * u0[1] + CV[i][2] * u0[2];
            const double uu = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
            const double fe = (double)weight(i) * rho0 * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu);
            f[i] = fe * (1.0 + 0.02 * (2 * U(rng) - 1));
        }
        bool outside = false;
        for (int i = 0; i < 19; i++) outside |= !(f[i] >= 0x1p-6 && f[i] < 16.0);
        fallback_states += outside;
        LD rho = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < 19; i++) {
            rho += f[i];
            for (int a = 0; a < 3; a++) j[a] += (LD)CV[i][a] * f[i];
        }
        LD u[3], uu = 0, uF = 0;
        for (int a = 0; a < 3; a++) {
            u[a] = (j[a] + 0.5L * F[a]) / rho;
            uu += u[a] * u[a];
            uF += u[a] * F[a];
        }
        LD ref[19], mass_in = 0, mass_ref = 0;
        for (int i = 0; i < 19; i++) {
            const LD cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
            const LD cF = CV[i][0] * (LD)F[0] + CV[i][1] * (LD)F[1] + CV[i][2] * (LD)F[2];
            const LD feq = weight(i) * rho * (1 + 3 * cu + 4.5L * cu * cu - 1.5L * uu);
            const LD S = (LD)beta * weight(i) * (3 * cF - 3 * uF + 9 * cu * cF);
            ref[i] = (1 - (LD)omega) * f[i] + (LD)omega * feq + S;
            mass_in += f[i];
            mass_ref += ref[i];
        }
        // both ways of forming the force terms: per launch (uniform force) and per node
        for (int way = 0; way < 2; way++) {
            double g[19];
            for (int i = 0; i < 19; i++) g[i] = f[i];
            collide_df<false>(g, F[0], K, way == 0);
            LD mass_out = 0;
            for (int i = 0; i < 19; i++) {
                coll_abs = std::fmax(coll_abs, (double)(fabsl((LD)g[i] - ref[i]) / weight(i)));
                mass_out += g[i];
            }
            mass_rel = std::fmax(mass_rel, (double)(fabsl(mass_out - mass_in) / mass_in));
        }
    }
    std::printf("collide_abs_over_w %.3e\n", coll_abs);
    std::printf("collide_mass_rel %.3e\n", mass_rel);
    std::printf("collide_fallback_states %ld\n", fallback_states);

    // the incompressible form (INC): f^eq = w (rho + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u), u = j + F/2,
    // and the Guo term with that u
    double inc_abs = 0;
    for (int n = 0; n < 100000; n++) {
        const double tau = 0.51 + 1.5 * U(rng), omega = 1.0 / tau, beta = 1.0 - 0.5 / tau;
        const double F[3] = {1e-4 * (2 * U(rng) - 1), 1e-4 * (2 * U(rng) - 1), 1e-4 * (2 * U(rng) - 1)};
        const DFConst K = make_df_const(omega, beta, F[0], F[1], F[2]);
        double f[19];
        const double u0[3] = {0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1)};
        const double rho0 = 0.95 + 0.1 * U(rng);
        for (int i = 0; i < 19; i++) {
            const double cu = CV[i][0] * u0[0] + CV[i][1] * u0[1] + CV[i][2] * u0[2];
            f[i] = (double)weight(i) * (rho0 + 3 * cu) * (1.0 + 0.02 * (2 * U(rng) - 1));
        }
        LD rho = 0, u[3] = {0, 0, 0};
        for (int i = 0; i < 19; i++) {
            rho += f[i];
            for (int a = 0; a < 3; a++) u[a] += (LD)CV[i][a] * f[i];
        }
        LD uu = 0, uF = 0;
        for (int a = 0; a < 3; a++) {
            u[a] += 0.5L * F[a];
            uu += u[a] * u[a];
            uF += u[a] * F[a];
        }
        for (int way = 0; way < 2; way++) {
            double g[19];
            for (int i = 0; i < 19; i++) g[i] = f[i];
            collide_df<false, true>(g, F[0], K, way == 0);
            for (int i = 0; i < 19; i++) {
                const LD cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
                const LD cF = CV[i][0] * (LD)F[0] + CV[i][1] * (LD)F[1] + CV[i][2] * (LD)F[2];
                const LD feq = weight(i) * (rho + 3 * cu + 4.5L * cu * cu - 1.5L * uu);
                const LD S = (LD)beta * weight(i) * (3 * cF - 3 * uF + 9 * cu * cF);
                const LD ref = (1 - (LD)omega) * f[i] + (LD)omega * feq + S;
                inc_abs = std::fmax(inc_abs, (double)(fabsl((LD)g[i] - ref) / weight(i)));
            }
        }
    }
    std::printf("collide_inc_abs_over_w %.3e\n", inc_abs);

    // closure_df: inlet f^eq(rho, u_in) and outlet f^eq(rho_out, (j + F/2) / rho) against
    // long double, with a uniform and a per-node F_x
    double close_abs = 0;
    for (int n = 0; n < 100000; n++) {
        const double tau = 0.51 + 1.5 * U(rng), omega = 1.0 / tau, beta = 1.0 - 0.5 / tau;
        const double F[3] = {1e-4 * (2 * U(rng) - 1), 1e-4 * (2 * U(rng) - 1), 1e-4 * (2 * U(rng) - 1)};
        const double uin[3] = {0.1 * (2 * U(rng) - 1), 0.05 * (2 * U(rng) - 1), 0.05 * (2 * U(rng) - 1)};
        const double rho_out = 0.95 + 0.1 * U(rng);
        const DFConst K = make_df_const(omega, beta, F[0], F[1], F[2]);
        const DFClosure Bc = make_df_closure(uin, rho_out);
        double f[19];
        const double u0[3] = {0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1)};
        for (int i = 0; i < 19; i++) {
            const double cu = CV[i][0] * u0[0] + CV[i][1] * u0[1] + CV[i][2] * u0[2];
            f[i] = (double)weight(i) * (1 + 3 * cu) * (1.0 + 0.02 * (2 * U(rng) - 1));
        }
        LD rho = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < 19; i++) {
            rho += f[i];
            for (int a = 0; a < 3; a++) j[a] += (LD)CV[i][a] * f[i];
        }
        for (int type = 2; type <= 3; type++) {
            LD r, u[3];
            for (int a = 0; a < 3; a++) u[a] = type == 2 ? (LD)uin[a] : (j[a] + 0.5L * F[a]) / rho;
            r = type == 2 ? rho : (LD)rho_out;
            const LD uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            for (int way = 0; way < 2; way++) {
                double g[19];
                for (int i = 0; i < 19; i++) g[i] = f[i];
                closure_df(g, type, F[0], K, Bc, way == 0);
                for (int i = 0; i < 19; i++) {
                    const LD cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
                    const LD feq = weight(i) * r * (1 + 3 * cu + 4.5L * cu * cu - 1.5L * uu);
                    close_abs = std::fmax(close_abs, (double)(fabsl((LD)g[i] - feq) / weight(i)));
                }
            }
        }
    }
    std::printf("closure_abs_over_w %.3e\n", close_abs);

    // the form for a force along x (F_y = F_z = 0) against the general form, bit for bit,
    // with a uniform and a per-node F_x, F_x = 0 included
    long xf_mismatch = 0;
    for (int n = 0; n < 100000; n++) {
        const double tau = 0.51 + 1.5 * U(rng), omega = 1.0 / tau, beta = 1.0 - 0.5 / tau;
        const double Fx = n % 10 == 0 ? 0.0 : 1e-4 * (2 * U(rng) - 1);
        const DFConst K = make_df_const(omega, beta, Fx, 0.0, 0.0);
        double f[19];
        const double u0[3] = {0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1), 0.1 * (2 * U(rng) - 1)};
        for (int i = 0; i < 19; i++) {
            const double cu = CV[i][0] * u0[0] + CV[i][1] * u0[1] + CV[i][2] * u0[2];
            f[i] = (double)weight(i) * (1 + 3 * cu) * (1.0 + 0.02 * (2 * U(rng) - 1));
        }
        for (int way = 0; way < 2; way++) {
            double a[19], b[19];
            for (int i = 0; i < 19; i++) a[i] = b[i] = f[i];
            collide_df<false>(a, Fx, K, way == 0);
            collide_df<true>(b, Fx, K, way == 0);
            for (int i = 0; i < 19; i++)
                if (std::memcmp(&a[i], &b[i], sizeof(double)) != 0) xf_mismatch++;
        }
    }
    std::printf("collide_xf_mismatches %ld\n", xf_mismatch);
    return 0;
}
