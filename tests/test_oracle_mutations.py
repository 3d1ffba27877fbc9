"""Plant plausible mistakes in a copy of the oracle and check that its pins catch each.

Every mutant is one textual change to ``oracle/oracle.c`` (a dropped term, a wrong
sign, coefficient, index or operand), compiled into a throw-away library and run
against the pin battery below in a child process. A mutant that passes every pin
would mean the pins leave that part of the oracle unchecked.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = [
    ("feq quadratic coefficient", "rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);\n}",
     "rho * (1.0 + 3.0 * cu + 4.0 * cu * cu - 1.5 * uu);\n}"),
    ("feq u^2 sign", "rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);\n}", "rho * (1.0 + 3.0 * cu + 4.5 * cu * cu + 1.5 * uu);\n}"),
    ("feq linear coefficient", "(1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);\n}", "(1.0 + 2.0 * cu + 4.5 * cu * cu - 1.5 * uu);\n}"),
    ("Guo prefactor", "return (1.0 - 0.5 / tau) * W[i]", "return (1.0 - 1.0 / tau) * W[i]"),
    ("Guo u.F sign", "3.0 * (cF - uF) + 9.0 * cu * cF);\n}", "3.0 * (cF + uF) + 9.0 * cu * cF);\n}"),
    ("Guo second-order term dropped", "3.0 * (cF - uF) + 9.0 * cu * cF);\n}", "3.0 * (cF - uF) + 0.0 * cu * cF);\n}"),
    ("half-force velocity shift dropped",
     "u[a] = (j[a] + 0.5 * F[a]) / rho;\n    if (type == INLET)", "u[a] = (j[a] + 0.0 * F[a]) / rho;\n    if (type == INLET)"),
    ("BGK relaxation time", "out[i] = f[i] - (f[i] - feq(i, rho, u)) / tau + guo", "out[i] = f[i] - (f[i] - feq(i, rho, u)) / (tau + 0.1) + guo"),
    ("inlet density", "out[i] = feq(i, rho, u_in);", "out[i] = feq(i, 1.0, u_in);"),
    ("outlet density", "out[i] = feq(i, rho_out, u);", "out[i] = feq(i, rho, u);"),
    ("bounce-back takes own direction",
     "f[i] = A[opp(i) * N + n];\n                }\n                force_at(n, g, g_field, F);\n                oracle_collide(f,",
     "f[i] = A[i * N + n];\n                }\n                force_at(n, g, g_field, F);\n                oracle_collide(f,"),
    ("push instead of pull", "int p[3] = {x - C[i][0], y - C[i][1], z - C[i][2]};", "int p[3] = {x + C[i][0], y + C[i][1], z + C[i][2]};"),
    ("periodic wrap off by one", "p[a] = (p[a] + n[a]) % n[a];", "p[a] = (p[a] + n[a] + 1) % n[a];"),
    ("gather from solid nodes",
     "if (source_node(x, y, z, i, nx, ny, nz, periodic, &s) && nt[s] != SOLID)\n                        f[i] = A[i * N + s];\n"
     "                    else\n                        f[i] = A[opp(i) * N + n];\n                }\n                force_at(n, g, g_field, F);\n"
     "                oracle_collide(f,",
     "if (source_node(x, y, z, i, nx, ny, nz, periodic, &s))\n                        f[i] = A[i * N + s];\n"
     "                    else\n                        f[i] = A[opp(i) * N + n];\n                }\n                force_at(n, g, g_field, F);\n"
     "                oracle_collide(f,"),
    ("diagonal weight", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 35.0};"),
    ("velocity table", "{0, -1, 1}, {0, -1, -1}};", "{0, -1, 1}, {0, 1, -1}};"),
    ("reported velocity shift sign", "u[a * N + n] = (j[a] - 0.5 * F[a]) / r;", "u[a * N + n] = (j[a] + 0.5 * F[a]) / r;"),
    ("reduced momentum shift sign", "p[a] += j[a] - 0.5 * F[a];", "p[a] += j[a] + 0.5 * F[a];"),
    ("tiling drops boundary-only tiles", "if (nt[x + (long)nx * (y + (long)ny * z)] != SOLID) keep = 1;",
     "if (nt[x + (long)nx * (y + (long)ny * z)] == FLUID) keep = 1;"),
    ("tiling index order", "long t = tx + (long)Tx * (ty + (long)Ty * tz);\n                int keep",
     "long t = ty + (long)Ty * (tx + (long)Tx * tz);\n                int keep"),
    ("tiled slot transposed", "src_s = (sx & 3) + 4 * (sy & 3) + 16 * (sz & 3);", "src_s = (sy & 3) + 4 * (sx & 3) + 16 * (sz & 3);"),
    ("adjoint: relaxation factor dropped", "mu[i] += lam[i] * (1.0 - 1.0 / tau);", "mu[i] += lam[i];"),
    ("adjoint: half-force term", "Fbar[a] += 0.5 * ubar[a] / rho;", "Fbar[a] += ubar[a] / rho;"),
    ("adjoint: bounce-back transpose", "lam[opp(i) * N + n] += mu[i];", "lam[i * N + n] += mu[i];"),
    ("adjoint: Guo prefactor derivative", "lam[i] * W[i] * qi * 0.5 / (tau * tau);", "lam[i] * W[i] * qi * 0.5 / tau;"),
    ("loss seed sign", "lam[i * N + n] = (C[i][0] - ux) / r / (double)count;", "lam[i * N + n] = (C[i][0] + ux) / r / (double)count;"),
    ("tangent quotient rule", "(a.d * b.v - a.v * b.d) / (b.v * b.v)", "(a.d * b.v + a.v * b.d) / (b.v * b.v)"),
    ("MRT energy row", "case 1: return 19.0 * cc - 30.0;", "case 1: return 19.0 * cc - 29.0;"),
    ("MRT q row", "case 4: return (5.0 * cc - 9.0) * x;", "case 4: return (5.0 * cc - 8.0) * x;"),
    ("MRT m_y row component", "case 17: return (z * z - x * x) * y;", "case 17: return (z * z - x * x) * x;"),
    ("MRT force factor", "(1.0 - 0.5 * rates[k]) * mG", "(1.0 - rates[k]) * mG"),
    ("MRT relaxes towards m", "mstar[k] = (m - rates[k] * (m - meq)", "mstar[k] = (m - rates[k] * (meq - m)"),
    ("MRT inverse without norm", ") * mG) / norm;", ") * mG) / 1.0;"),
    ("incompressible feq linear term", "return W[i] * (rho + 3.0 * cu", "return W[i] * (rho + 3.0 * rho * cu"),
    ("incompressible velocity divides by rho", "? (j[a] + 0.5 * F[a]) / rho : j[a] + 0.5 * F[a];",
     "? (j[a] + 0.5 * F[a]) / rho : (j[a] + 0.5 * F[a]) / rho;"),
    ("incompressible reported velocity", "u[a * N + n] = j[a] - 0.5 * F[a];", "u[a * N + n] = j[a] + 0.5 * F[a];"),
    ("moving wall term sign", "f[i] += 6.0 * W[i] * (C[i][0] * lid_u[0]", "f[i] -= 6.0 * W[i] * (C[i][0] * lid_u[0]"),
    ("moving wall term factor", "f[i] += 6.0 * W[i] * (C[i][0] * lid_u[0]", "f[i] += 3.0 * W[i] * (C[i][0] * lid_u[0]"),
    ("moving wall on the opposite face", "return (face % 2 == 0) ? q < 0 : q >= n;", "return (face % 2 == 1) ? q < 0 : q >= n;"),
    ("Zou-He axis term", "v += jn / 3.0;", "v += jn / 6.0;"),
    ("Zou-He transverse correction sign", "v += (jn + t * j[tang]) / 6.0 - t * N;", "v += (jn + t * j[tang]) / 6.0 + t * N;"),
    ("Zou-He outgoing sum counted once", "B += 2.0 * f[i];", "B += f[i];"),
    ("Zou-He velocity density", "rho = eq == 0 ? B / (1.0 - un) : B + un;", "rho = eq == 0 ? B / (1.0 + un) : B + un;"),
    ("model step bounce-back", "f[i] = A[opp(i) * N + n];\n                        if (beyond_face(",
     "f[i] = A[i * N + n];\n                        if (beyond_face("),
]


def _battery():
    """Pins in order of cost; returns the name of the first that fails, or None."""
    import test_oracle_adjoint as A
    import test_oracle_models as Mo
    import test_oracle_pins as P
    checks = [
        ("lattice constants", P.test_lattice_matches_paper_constants),
        ("lattice isotropy", P.test_lattice_isotropy),
        ("collision moments", lambda: [P.test_collision_moments_fluid(s) for s in range(2)]),
        ("single relaxation", lambda: P.test_collision_single_relaxation_rate(0)),
        ("boundary closures", P.test_collision_boundary_closures),
        ("tiling golden", P.test_tiling_channel8_golden),
        ("tiling brute force", lambda: [P.test_tiling_brute_force(s) for s in range(4)]),
        ("equilibrium fixed point", P.test_equilibrium_fixed_point_with_walls),
        ("uniform flow fixed point", P.test_uniform_flow_fixed_point_periodic),
        ("mass", lambda: P.test_mass_conservation(1e-4)),
        ("momentum closed form", P.test_momentum_closed_form),
        ("uniform acceleration", P.test_uniform_acceleration_closed_form),
        ("streaming shift", P.test_streaming_is_shift_when_collision_off),
        ("time reversal", P.test_streaming_time_reversal_with_walls),
        ("dense vs tiled", lambda: [P.test_dense_and_tiled_bit_identical(p) for p in (0, 7, 5)]),
        ("tangent vs FD", lambda: A.test_tangent_matches_central_differences(0b111)),
        ("dot product", lambda: [A.test_adjoint_dot_product(p) for p in (0, 7)]),
        ("loss gradient", lambda: A.test_loss_gradient_matches_fd(True)),
        ("shear wave", P.test_shear_wave_decay_rate),
        ("Poiseuille", P.test_poiseuille_closed_form),
        ("MRT basis", Mo.test_basis_orthogonal_with_published_norms),
        ("equilibrium moments", lambda: [Mo.test_equilibrium_moments_match_published_closed_forms(e) for e in (0, 1)]),
        ("MRT = LBGK", lambda: [Mo.test_mrt_with_equal_rates_is_lbgk(e) for e in (0, 1)]),
        ("incompressible LBGK", Mo.test_lbgk_incompressible_from_collide_m_matches_definition),
        ("single moment", lambda: [Mo.test_single_moment_relaxes_by_its_own_rate(k) for k in (1, 2, 4, 9, 10, 16)]),
        ("MRT conservation", lambda: [Mo.test_mrt_conserves_mass_and_adds_force(e) for e in (0, 1)]),
        ("incompressible momentum", lambda: [Mo.test_incompressible_momentum_closed_form(c) for c in (0, 1)]),
        ("magic Poiseuille", lambda: [Mo.test_poiseuille_exact_at_magic_lambda(e, c) for e in (0, 1) for c in (0, 1)]),
        ("Couette", lambda: Mo.test_couette_exact_with_moving_lid(0.8, 0)),
        ("Zou-He moments", lambda: [Mo.test_zou_he_reconstruction_sets_density_and_momentum(fc, e)
                                    for fc in range(6) for e in (0, 1)]),
        ("Zou-He fixed point", lambda: [Mo.test_zou_he_uniform_flow_is_a_fixed_point((0, 1), e) for e in (0, 1)]),
    ]
    for name, fn in checks:
        try:
            fn()
        except Exception:
            return name
    return None


def _compile(text, out):
    with open(out + ".c", "w") as fh:
        fh.write(text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-w", out + ".c", "-o", out, "-lm"], check=True)


def _run_mutant(args):
    k, name, text, td = args
    so = os.path.join(td, f"m{k}.so")
    _compile(text, so)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), so], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    caught = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else f"exit {r.returncode}"
    return name, r.returncode == 0 and caught == "SURVIVED"


def test_every_mutant_is_caught():
    from concurrent.futures import ThreadPoolExecutor
    src = open(SRC).read()
    for name, old, _ in MUTANTS:
        assert src.count(old) == 1, f"mutation site not unique: {name}"
    with tempfile.TemporaryDirectory() as td:
        jobs = [(k, name, src.replace(old, new), td) for k, (name, old, new) in enumerate(MUTANTS)]
        # each mutant compiles and runs in its own child process: run them side by side
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(_run_mutant, jobs))
    survivors = [name for name, survived in results if survived]
    assert not survivors, f"mutants not caught by any pin: {survivors}"


if __name__ == "__main__":
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import oracle as O
    O._lib = O.load(sys.argv[1])
    failed = _battery()
    print("SURVIVED" if failed is None else f"CAUGHT by {failed}")
