"""Pins of the oracle's mean-field potential and energy functional (Sec. 4.3, eq:ham_tdhf
in the density-dependent form V = V_ext + a rho + b rho^(1+alpha)), shared by the pin
tests and by the planted-mistake tests, which run them on a mutated copy of ``System``.

Neither pin retypes the oracle's formulas:

* ``energy_drift``: with zero Dirichlet faces the exact mean-field dynamics conserves
  E[phi] exactly when V = dE/drho.  The stepper holds V at the step's start density, so
  a step changes E by O(dt^2) and a run of fixed length T by O(dt): halving dt must halve
  the change, and its Richardson extrapolation to dt -> 0 must vanish.  A potential that
  is not the derivative of the functional (a wrong power, a missing orbital sum, a stray
  weight, a wrong coefficient on either side) changes E at a rate that does not shrink
  with dt.
* ``potential_scaling``: properties of the density dependence that hold for any state:
  with b = 0 the potential is linear in the density and the density is additive over
  orbitals; with a = 0 scaling every orbital by c scales V - V_ext by c^(2 (1+alpha));
  V does not depend on the grid spacing for the same node values.
* ``energy_scaling``: E - E_linear scales by c^4 (b = 0) and by c^(2 (2+alpha)) (a = 0).
"""
from __future__ import annotations

import numpy as np

from oracle.lattice import Box
from paper_1908_02456_gb300 import inputs

MF_STRONG = (-30.0, 20.0, 1.0 / 6.0)     # strong enough that V(rho) moves the orbitals


def small_case(b=3, N=8, h=0.5, seed=5):
    box = Box((N,) * 3, h)
    psi = inputs.orbital_set((N,) * 3, h, np.random.default_rng(seed), b).reshape(b, -1)
    return box, psi


def energy_drift(system_cls, T=0.4, dts=(0.01, 0.005), mf=MF_STRONG):
    """Change of E over a run of length T for each dt (zero Dirichlet faces)."""
    box, psi = small_case()
    out = []
    for dt in dts:
        sy = system_cls(box, meanfield=mf)
        e0 = sy.energy_functional(psi)
        phi, _, _ = sy.run(psi, dt, int(round(T / dt)))
        out.append(sy.energy_functional(phi) - e0)
    return out


def energy_drift_ok(system_cls) -> bool:
    d1, d2 = energy_drift(system_cls)
    ratio = d1 / d2
    richardson = 2.0 * d2 - d1
    return 1.8 < ratio < 2.2 and abs(richardson) < 0.03 * abs(d1)


def potential_scaling_ok(system_cls) -> bool:
    box, psi = small_case()
    alpha = 1.0 / 6.0
    Vext = np.linspace(-0.3, 0.4, box.n)
    ok = True
    # b = 0: linear in the density, and the density adds over orbitals
    lin = system_cls(box, V_ext=Vext, meanfield=(-2.0, 0.0, alpha))
    parts = sum(lin.potential(psi[j:j + 1]) - Vext for j in range(psi.shape[0]))
    ok &= np.allclose(lin.potential(psi) - Vext, parts, rtol=1e-12, atol=0)
    ok &= np.allclose(lin.potential(1.7 * psi) - Vext, 1.7 ** 2 * (lin.potential(psi) - Vext), rtol=1e-12)
    # a = 0: homogeneous of degree 2 (1 + alpha) in the orbitals
    pw = system_cls(box, V_ext=Vext, meanfield=(0.0, 0.9, alpha))
    c = 1.3
    ok &= np.allclose(pw.potential(c * psi) - Vext, c ** (2 * (1 + alpha)) * (pw.potential(psi) - Vext),
                      rtol=1e-12)
    # no dependence on the grid spacing for the same node values
    other = system_cls(Box(box.shape[::-1], 0.8 * box.h), V_ext=Vext, meanfield=(-1.0, 0.8, alpha))
    same = system_cls(box, V_ext=Vext, meanfield=(-1.0, 0.8, alpha))
    ok &= np.allclose(other.potential(psi), same.potential(psi), rtol=1e-13)
    return bool(ok)


def energy_scaling_ok(system_cls) -> bool:
    box, psi = small_case()
    alpha = 1.0 / 6.0
    linear = system_cls(box)

    def e_int(sy, p):
        return sy.energy_functional(p) - linear.energy_functional(p)
    ok = True
    c = 1.3
    sa = system_cls(box, meanfield=(-2.0, 0.0, alpha))
    ok &= np.isclose(e_int(sa, c * psi), c ** 4 * e_int(sa, psi), rtol=1e-12)
    sb = system_cls(box, meanfield=(0.0, 0.9, alpha))
    ok &= np.isclose(e_int(sb, c * psi), c ** (2 * (2 + alpha)) * e_int(sb, psi), rtol=1e-12)
    ok &= abs(e_int(sa, psi)) > 1e-3 and abs(e_int(sb, psi)) > 1e-3
    return bool(ok)
