"""TEBD on the GPU reaches the ground energy of the open critical transverse-field
Ising chain (L = 64, chi = 128): the free-fermion closed form
E0 = 1 - 1/sin(pi / (2 (2L + 1))) = -81.12598012314353 (stored in
tests/golden/tfim_critical_e0.json), within 1e-6 relative - the bound set by
the second-order Trotter error at the final dt (energy error ~ dt^4) and the
bond-dimension truncation.  Imaginary-time schedule dt = 0.1, 0.05, 0.02 as in
the paper's protocol of reducing dt (Sec. III.C)."""
import json
import os

import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import tebd as otebd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tebd_l64_reaches_free_fermion_energy():
    need_gpu()
    from paper_1710_01463_gb300 import tebd
    e0 = json.load(open(os.path.join(HERE, "golden", "tfim_critical_e0.json")))["energies"]["64"]["closed_form"]
    L = 64
    ch = tebd.TebdChain(L, 128, h=1.0, p=10, q=2, seed=11)
    ch.set_product_state(inputs.product_state_vectors(L, 2, 102))
    step = 0
    for dt, n in ((0.1, 700), (0.05, 500), (0.02, 250)):
        ch.set_dt(dt)
        for _ in range(n):
            ch.step(step)
            step += 1
    torch.cuda.synchronize()
    assert int((ch.info[..., 0] < 0).sum()) == 0
    e = otebd.mps_energy(ch.tensors(), L, 1.0)
    rel = (e - e0) / abs(e0)
    assert 0.0 <= rel < 1e-6, rel
    lam = ch.schmidt_values()
    for j in range(1, L):
        assert abs(np.sum(lam[j] ** 2) - 1.0) < 1e-12
