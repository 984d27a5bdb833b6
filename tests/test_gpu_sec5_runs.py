"""The Langmuir (X5) and gyration (X6) runs of Sec. 5 (Fig. 3) through the
library, at test sizes, against what the physics fixes:

- X5: every electron carries the same directed momentum against immovable
  ions, so the plasma oscillates as a whole: the field energy oscillates with
  period pi/omega, omega = omega_pe / gamma^(3/2) for the longitudinal motion
  at 0.1c, while the total energy integral stays within the scheme's small
  defect (the paper: about 1e-5).
- X6: an electron and a positron gyrate in a uniform B_z with
  omega_Be dt = 0.25; the Larmor radius is w c / (|q| B / m) and the kinetic
  energy decreases only slowly (the paper: a small gradual decrease).
"""
import math

import pytest

from paper_1101_0809_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1101_0809_gb300 import build as B
    B.build()
    from paper_1101_0809_gb300 import pic
    return pic


def test_x5_langmuir_period_and_energy(P):
    from paper_1101_0809_gb300.energy import energy_run, oscillation_period
    wl, bx = W.x5_langmuir(n=16, steps=400, tile=(4, 4, 4))
    r = energy_run(wl, 3, P.PIC_FP64, every=2, bx=bx)
    steps = [s[0] for s in r["series"]]
    fe = [s[3] for s in r["series"]]
    period = oscillation_period(steps, fe)
    gam = math.sqrt(1.0 + (2.0 / wl.c) ** 2)          # the stream: w = 2 v_th = 0.1c
    expect = math.pi * gam ** 1.5 / wl.dt              # in steps, omega_pe = 1
    assert period == pytest.approx(expect, rel=0.03), (period, expect)
    assert max(fe) > 10 * fe[0]                        # the oscillation is there
    assert r["max_rel_defect"] < 1e-4


def test_x6_gyration_radius_and_slow_energy_loss(P):
    from paper_1101_0809_gb300.energy import gyration_run
    wl, bz = W.x6_gyration(n=16, steps=400, tile=(4, 4, 4))
    r = gyration_run(wl, 3, P.PIC_FP64, bz)
    larmor = 0.5 * wl.c * wl.c / bz                    # w c / B with w = 0.5c, |q| = m = 1
    assert r["larmor_radius_first"] == pytest.approx(larmor, rel=0.05)
    assert 0.95 < r["kinetic_ratio"] <= 1.0 + 1e-6
    assert r["larmor_radius_last"] <= r["larmor_radius_first"] * (1 + 1e-3)
