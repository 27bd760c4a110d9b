"""The symmetry relabelling used to augment the warm-start network's training data.

Transport commutes with the cube's symmetries: relabelling the template and
the velocity by an element g (axes permuted and flipped, velocity components
permuted with the axes and negated along flipped axes) must relabel m(1) the
same way.  The discrete scheme keeps this exactly: under i -> n - 1 - i the
node set {floor(q) - 1, .., floor(q) + 2} of a departure point q maps onto the
node set of the mirrored point, so the cubic interpolant is the same and the
FP64 oracle's transport of the relabelled pair reproduces the relabelled m(1)
to rounding.  A wrong component rule leaves an O(1) difference.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import transport as OT
from paper_2401_17493_b300 import synth
from paper_2401_17493_b300.unet import symmetry

N = 32


def _case():
    m0, _, _ = synth.blob_pair((N, N, N), seed=8, kmax=2, max_disp_voxels=1.0)
    v = synth.bandlimited_velocity((N, N, N), 2, 1.5, 9)
    m1 = OT.state_solve(m0.astype(np.float64), v, 4)[-1]
    return m0.astype(np.float64), v, m1


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("g", [1, 7, 8, 21, 42, 47])
def test_relabelled_pair_transports_to_the_relabelled_image(g):
    m0, v, m1 = _case()
    fields = torch.from_numpy(np.stack([m0, m1]))
    f, vg = symmetry(fields, torch.from_numpy(v), g)
    m0g, m1g = f[0].numpy(), f[1].numpy()
    out = OT.state_solve(m0g, vg.numpy(), 4)[-1]
    assert _rel(out, m1g) < 1e-12


def test_identity_element_changes_nothing():
    m0, v, m1 = _case()
    fields = torch.from_numpy(np.stack([m0, m1]))
    f, vg = symmetry(fields, torch.from_numpy(v), 0)
    assert torch.equal(f, fields) and torch.equal(vg, torch.from_numpy(v))


def test_a_wrong_component_rule_is_far_off():
    m0, v, m1 = _case()
    fields = torch.from_numpy(np.stack([m0, m1]))
    f, vg = symmetry(fields, torch.from_numpy(v), 5)          # flips of axes 0 and 2
    wrong = vg.clone()
    wrong[0] = -wrong[0]                                      # forget one sign
    out = OT.state_solve(f[0].numpy(), wrong.numpy(), 4)[-1]
    assert _rel(out, f[1].numpy()) > 2e-2
