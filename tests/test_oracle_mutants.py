"""Planted mistakes in the CPU oracle, each caught by one of its pins.

For every entry below the oracle's C source is copied, one fragment is
replaced by a plausible mistake (a dropped term, a wrong sign, average,
coefficient or index), the copy is compiled into a library of its own, and
the named pin is run against that library: it must fail.  The oracle source
itself is never changed; the fragment must occur exactly once, so a later
edit of the oracle that moves it makes this test fail loudly instead of
passing vacuously.
"""
import contextlib
import os
import subprocess

import pytest

from oracle import oracle as O
from tests import test_oracle_pins as P

MUTANTS = [
    # characteristic WENO flux: one Lax-Friedrichs alpha for all fields
    ("global LLF alpha",
     "for (int m = 0; m < np; ++m) alpha = fmax(alpha, fabs(lam[m][e]));",
     "for (int m = 0; m < np; ++m) for (int ee = 0; ee < 5; ++ee) alpha = fmax(alpha, fabs(lam[m][ee]));",
     lambda: P.test_weno_entropy_wave_linear_upwind_symbol(5, 0.6)),
    # Roe state: arithmetic-mean total enthalpy
    ("arithmetic-mean Roe enthalpy",
     "out[3] = (ra * H[0] + rb * H[1]) / (ra + rb);",
     "out[3] = 0.5 * (H[0] + H[1]);",
     P.test_roe_average_property_calorically_perfect),
    # Roe state: arithmetic-mean velocity
    ("arithmetic-mean Roe velocity",
     "for (int a = 0; a < 3; ++a) out[a] = (ra * sa[1 + a] + rb * sb[1 + a]) / (ra + rb);",
     "for (int a = 0; a < 3; ++a) out[a] = 0.5 * (sa[1 + a] + sb[1 + a]);",
     P.test_roe_average_property_calorically_perfect),
    # WENO minus flux taken from the wrong side
    ("minus flux not mirrored",
     "int mm = np - 1 - m;",
     "int mm = m + 1;",
     lambda: P.test_weno_acoustic_wave_linear_upwind_symbol(5, -1)),
    # WENO5 optimal weights reversed
    ("WENO5 optimal weights reversed",
     "static const double WENO5_D[3] = {0.1, 0.6, 0.3};",
     "static const double WENO5_D[3] = {0.3, 0.6, 0.1};",
     lambda: P.test_weno_entropy_wave_linear_upwind_symbol(5, 0.6)),
    # WENO7 smoothness indicator coefficient
    ("WENO7 indicator coefficient",
     "b[k] = 240.0 * s1 * s1 + 260.0 * s2 * s2 + 781.0 / 3.0 * e3 * e3;",
     "b[k] = 240.0 * s1 * s1 + 270.0 * s2 * s2 + 781.0 / 3.0 * e3 * e3;",
     lambda: P.test_weno_smoothness_indicators_and_weights(7)),
    # eigenvector sign
    ("left eigenvector sign",
     "Lm[1 * 5 + 0] = 1.0 - b * q2 / (2.0 * c2);",
     "Lm[1 * 5 + 0] = 1.0 + b * q2 / (2.0 * c2);",
     lambda: P.test_eigenvectors_diagonalise_jacobian(0)),
    # split-form central flux: pressure mean dropped
    ("central flux pressure dropped",
     "pp += s->p[a] + s->p[b];",
     "pp += 2.0 * s->p[a];",
     lambda: P.test_kinetic_energy_preservation(6)),
    # split-form central flux: factor 2 of the double sum dropped
    ("central flux factor 2",
     "for (int f = 0; f < 5; ++f) F[f] += 2.0 * A1[l] * acc[f];",
     "for (int f = 0; f < 5; ++f) F[f] += A1[l] * acc[f];",
     lambda: P.test_modified_wavenumber_entropy_wave(0, 6)),
    # viscous terms: transposed gradient dropped
    ("viscous cross term dropped",
     "for (int b = 0; b < 3; ++b) m += gmu[b] * (g[a][b] + g[b][a]);",
     "for (int b = 0; b < 3; ++b) m += gmu[b] * (g[a][b] + g[a][b]);",
     lambda: P.test_design_order_manufactured(P._mms_exact(0.5, 100.0, 0.72, 1.4, 0.76), False, 6)),
    # isothermal wall ghost: temperature copied instead of mirrored about T_w
    ("wall temperature ghost",
     "s->T[a] = 2.0 * c->t_wall - s->T[b];",
     "s->T[a] = s->T[b];",
     P.test_design_order_manufactured_walls),
    # sensor: compressions and expansions swapped
    ("sensor sign",
     "double sv = -th / sqrt(th * th + om2 + s->eps_sensor);",
     "double sv = th / sqrt(th * th + om2 + s->eps_sensor);",
     P.test_sensor_closed_forms),
    # RK3 coefficient
    ("RK3 coefficient",
     "static const double RK_RHO[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};",
     "static const double RK_RHO[3] = {0.0, -17.0 / 60.0, -5.0 / 13.0};",
     P.test_rk3_third_order_and_consistency),
    # KEEP: arithmetic instead of logarithmic mean density
    ("KEEP arithmetic-mean density",
     "double rl = log_mean(s->rho[a], s->rho[b], s->c->keep);",
     "double rl = 0.5 * (s->rho[a] + s->rho[b]);",
     lambda: P.test_keep_conserves_entropy(6, False)),
    # KEEP: pressure work without the cross products
    ("KEEP pressure work",
     "0.5 * (s->p[a] * un[b] + s->p[b] * un[a]);",
     "0.5 * (s->p[a] * un[a] + s->p[b] * un[b]);",
     lambda: P.test_keep_conserves_entropy(6, False)),
    # KEEP: internal energy from the arithmetic mean of 1/T
    ("KEEP internal-energy mean",
     "double bl = log_mean(1.0 / s->T[a], 1.0 / s->T[b], s->c->keep); /* <1/T> */",
     "double bl = 0.5 * (1.0 / s->T[a] + 1.0 / s->T[b]);",
     lambda: P.test_keep_conserves_entropy(6, False)),
    # forcing: the work of the body force dropped from the energy equation
    ("forcing power dropped",
     "rhs[4 * n + q] += f * s->u[PI(s, i, j, k)];",
     "rhs[4 * n + q] += 0.0 * f;",
     P.test_forcing_is_body_force_with_its_power),
]


@contextlib.contextmanager
def _using(path):
    old = O._lib
    O._lib = O.load(path)
    try:
        yield
    finally:
        O._lib = old


def _build_mutant(tmp_path, idx, find, repl):
    src = open(O.SRC).read()
    assert src.count(find) == 1, "fragment must occur exactly once in the oracle: %r" % find
    path = os.path.join(str(tmp_path), "mutant%d.c" % idx)
    with open(path, "w") as f:
        f.write(src.replace(find, repl))
    lib = os.path.join(str(tmp_path), "libmutant%d.so" % idx)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", path, "-o",
                    lib, "-lm"], check=True)
    return lib


def test_unmutated_oracle_passes_the_selected_pins():
    """The pins used below pass on the oracle as it stands."""
    for _, _, _, pin in MUTANTS:
        pin()


@pytest.mark.parametrize("idx", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(tmp_path, idx):
    name, find, repl, pin = MUTANTS[idx]
    lib = _build_mutant(tmp_path, idx, find, repl)
    with _using(lib):
        with pytest.raises(AssertionError):
            pin()
