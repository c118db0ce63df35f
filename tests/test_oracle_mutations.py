"""The oracle's pins against planted mistakes.

Each case copies the oracle package, changes one expression of its C source
the way a plausible slip would (a dropped term, a wrong sign, a wrong index
or direction, a transposed operand, a wrong factor), builds the copy, and
runs the oracle's pin tests against it: at least one pin must fail.  A
control copy without change must pass them all, so the failures come from
the mutation and not from the harness."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_constants.py", "tests/test_oracle_step.py", "tests/test_oracle_fd.py",
        "tests/test_oracle_field.py", "tests/test_oracle_negative_eq.py"]

# name -> (exact original text, replacement); the original must occur once
MUTATIONS = {
    "alpha4 term dropped (Eq. WeqAlgo)":
        ("L->alpha4 * (b0 * eu) * (b0 * eu)", "0.0 * (b0 * eu) * (b0 * eu)"),
    "sign of the alpha3 term":
        ("+ L->alpha3 * b0 * eu +", "- L->alpha3 * b0 * eu +"),
    "alpha5 term without the 1/2":
        ("L->alpha5 * b0 * 0.5 * u2", "L->alpha5 * b0 * u2"),
    "beta0 dropped from alpha2":
        ("double alpha2 = L->A2_0 + L->A2_1 * b0 * eps;", "double alpha2 = L->A2_0 + L->A2_1 * eps;"),
    "alpha1 and alpha2 slopes swapped":
        ("double alpha1 = L->A1_0 + L->A1_1 * b0 * eps;", "double alpha1 = L->A1_0 + L->A2_1 * b0 * eps;"),
    "streaming to x - e_i (Eq. TransportStep)":
        ("int64_t t = shift_site(G, s, L->idx[i][0], L->idx[i][1], L->idx[i][2]);",
         "int64_t t = shift_site(G, s, -L->idx[i][0], -L->idx[i][1], -L->idx[i][2]);"),
    "energy about the origin, not u (Eq. DiscrAvr)":
        ("double c = L->xi * L->idx[i][k] - M->u[k];", "double c = L->xi * L->idx[i][k];"),
    "transposed off-diagonal of W (sign of s_y)":
        ("W->m[0][1] = 0.5 * (sx - I * sy);", "W->m[0][1] = 0.5 * (sx + I * sy);"),
    "relaxation rate tau/dt instead of dt/tau":
        ("double omega = dt / tau;", "double omega = tau / dt;"),
    "axis weight off by 1 %":
        ("else if (l1 == 1) L->w[q] = L->a;", "else if (l1 == 1) L->w[q] = 1.01 * L->a;"),
    "D3Q19 drops the edges instead of the corners":
        ("if (d == 3 && l1 == 3) continue;", "if (d == 3 && l1 == 2) continue;"),
    "lattice constant xi squared wrongly (2D)":
        ("L->xi = (3.0 / pi) * sqrt(3.0 * z3 / beta0);", "L->xi = (3.0 / pi) * sqrt(3.0 * z3) / beta0;"),
    "zeta: wrong alternating sign":
        ("double sgn = (k % 2 == 0) ? 1.0 : -1.0;", "double sgn = 1.0;"),
    "adjoint: (1 + omega) for (1 - omega)":
        ("Lout[i].m[j][k] *= (1.0 - omega);", "Lout[i].m[j][k] *= (1.0 + omega);"),
    "adjoint: rho cotangent without P_i":
        ("mat_axpy(&rhobar, omega * L->w[i] * P, &Lp[i]);", "mat_axpy(&rhobar, omega * L->w[i], &Lp[i]);"),
    "F_k integrand power s^(2k) for s^(2k+1)":
        ("return 2.0 * pow(s, 2.0 * k + 1.0) * fermi(s * s - x);", "return 2.0 * pow(s, 2.0 * k) * fermi(s * s - x);"),
    "FD energy without the factor d/2 (Eq. energyFDstdOmega)":
        ("double e = h / beta * (oracle_fd(h, beta * mu_up)", "double e = 1.0 / beta * (oracle_fd(h, beta * mu_up)"),
    "FD inversion: mu_dn from the larger eigenvalue":
        ("out[2] = species_nu(d, beta, ldn) / beta;", "out[2] = species_nu(d, beta, lup) / beta;"),
    "FD inversion: Bloch axis y component of the conjugate":
        ("out[4] = 2.0 * cimag(conj(v0) * v1);", "out[4] = -2.0 * cimag(conj(v0) * v1);"),
    "field: rotation of the wrong sense":
        ("U->m[0][0] = c - I * sn * bz;", "U->m[0][0] = c + I * sn * bz;"),
    "global energy without the 1/2 (Eq. GlobalTotalEnergy)":
        ("en += 0.5 * e2 * t;", "en += e2 * t;"),
    "global momentum without the lattice constant xi (Eq. GlobalVelocity)":
        ("double e = L.xi * L.idx[i][k];\n                mom[k] += e * t;",
         "double e = L.idx[i][k];\n                mom[k] += e * t;"),
    "velocity not divided by the density (Eq. DiscrAvr)":
        ("M->u[k] = (k < L->d) ? acc / M->n : 0.0;", "M->u[k] = (k < L->d) ? acc : 0.0;"),
    "eps0 in 3D: the two eta factors swapped (Eq. energyFDstdOmega)":
        ("1.5 * (1.0 - pow(2.0, -1.5)) * oracle_zeta(2.5) /\n               ((1.0 - pow(2.0, -0.5))",
         "1.5 * (1.0 - pow(2.0, -0.5)) * oracle_zeta(2.5) /\n               ((1.0 - pow(2.0, -1.5))"),
    "Pauli read-out: sign of s_y":
        ("*sy = creal(I * (W->m[0][1] - W->m[1][0]));", "*sy = creal(I * (W->m[1][0] - W->m[0][1]));"),
    "initial state ignores the given eps field":
        ("double e = eps ? eps[s] : eps0;", "double e = eps0;"),
    "adjoint: sign of d omega / d tau":
        ("double omega = dt / tau, dom_dtau = -dt / (tau * tau);",
         "double omega = dt / tau, dom_dtau = dt / (tau * tau);"),
    "FD density prefactor (pi/beta)^(d/2) for (2 pi/beta)^(d/2) (Eq. nFDstdOmega)":
        ("double h = 0.5 * d, pre = pow(2.0 * M_PI / beta, h);", "double h = 0.5 * d, pre = pow(M_PI / beta, h);"),
    "alpha2 term without the 1/2 of |e_i|^2/2 (Eq. WeqAlgo)":
        ("return alpha1 + alpha2 * b0 * 0.5 * e2 +", "return alpha1 + alpha2 * b0 * e2 +"),
    "equilibrium weighted by the rest weight w_0 in every direction":
        ("mat_axpy(&Weq[i], L->w[i] * poly_P(L, i, M->u, M->eps), &M->rho);",
         "mat_axpy(&Weq[i], L->w[0] * poly_P(L, i, M->u, M->eps), &M->rho);"),
    "diagonal weight of D3Q19 a/4 instead of a/2":
        ("else L->w[q] = (d == 2) ? L->a / 4.0 : L->a / 2.0;", "else L->w[q] = (d == 2) ? L->a / 4.0 : L->a / 4.0;"),
    "FD inversion: density scaled by (beta/pi)^(d/2) for (beta/2 pi)^(d/2)":
        ("double h = 0.5 * d, y = ns * pow(beta / (2.0 * M_PI), h);", "double h = 0.5 * d, y = ns * pow(beta / M_PI, h);"),
    "FD inversion: eigenvalue discriminant tr^2/2 for tr^2/4":
        ("double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));", "double disc = sqrt(fmax(0.5 * tr * tr - det, 0.0));"),
    "equilibrium eigenvalue: the larger one instead of the smaller":
        ("out[(int64_t)i * N + s] = 0.5 * (a + e) - sqrt(half * half + off * off);",
         "out[(int64_t)i * N + s] = 0.5 * (a + e) + sqrt(half * half + off * off);"),
    "equilibrium eigenvalue: off-diagonal entry dropped":
        ("double off = cabs(Weq[i].m[0][1]);", "double off = 0.0;"),
    "per-site field read from the wrong site's column":
        ("B[k] = field_B_site ? field_B_site[(int64_t)k * N + s] : field_B[k];",
         "B[k] = field_B_site ? field_B_site[(int64_t)k * N + (s + 1) % N] : field_B[k];"),
    "per-site field components transposed (x read as y)":
        ("B[k] = field_B_site ? field_B_site[(int64_t)k * N + s] : field_B[k];",
         "B[k] = field_B_site ? field_B_site[(int64_t)((k + 1) % 3) * N + s] : field_B[k];"),
    "adjoint read-out: sign of the s_y cotangent":
        ("o[2 * N] = 0.5 * creal(I * (Lo[i].m[0][1] - Lo[i].m[1][0]));",
         "o[2 * N] = -0.5 * creal(I * (Lo[i].m[0][1] - Lo[i].m[1][0]));"),
}


def run_pins(tmp_path, mutation):
    dst = tmp_path / "alt"
    dst.mkdir()
    shutil.copytree(os.path.join(ROOT, "oracle"), dst / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = dst / "oracle" / "qlbm_oracle.c"
    if mutation is not None:
        old, new = mutation
        text = src.read_text()
        assert text.count(old) == 1, "mutation site not found once: %r" % old
        src.write_text(text.replace(old, new))
    env = dict(os.environ, QLBM_ORACLE_DIR=str(dst))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r


def test_unmutated_copy_passes_the_pins(tmp_path):
    r = run_pins(tmp_path, None)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(tmp_path, name):
    r = run_pins(tmp_path, MUTATIONS[name])
    assert r.returncode == 1, "no pin caught: %s\n%s" % (name, r.stdout[-2000:])
