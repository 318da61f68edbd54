"""Named options through the C ABI: every settable option reads back what was set,
read-only ones refuse writes, and out-of-range values are DPD_EINVAL (no state change)."""
import numpy as np
import pytest

from paper_1807_09896_gb300 import dpd, inputs
from parity_helpers import make_system, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


SETTABLE = {
    "lambda": 0.55, "band_margin": 0.4, "reflect_variant": 1.0, "seed": 12345.0, "system": 7.0,
    "v_wall_x": 0.1, "v_wall_y": -0.2, "v_wall_z": 0.0, "shear_x": 0.03, "shear_y": -0.01,
    "shear_ref": 2.5, "sample_every": 3.0, "a_ff": 20.0, "a_fs": 30.0, "gamma": 3.0, "sigma": 2.0,
    "g_x": 0.01, "g_y": 0.0, "g_z": -0.02, "phase_eps": 0.6, "force_law": 1.0, "S_r_ff": 30.0,
    "S_a_ff": 15.0, "S_r_fs": 60.0, "S_a_fs": 30.0, "r0_r": 0.7, "r0_a": 0.95, "sph_dim": 2.0,
    "use_graph": 0.0, "graph_steps": 8.0, "force_variant": 2.0,
}
INVALID = {
    "reflect_variant": 2.0, "band_margin": 0.0, "seed": -1.0, "shear_z": 0.1, "shear_axis": 3.0,
    "force_law": 2.0, "r0_r": 1.5, "r0_a": 0.0, "sph_dim": 4.0, "phase_eps": 0.0,
    "graph_steps": 3.0, "force_variant": 1e6, "gamma": -1.0,
}


def test_options_round_trip_and_reject_bad_values():
    w = inputs.channel(6.0, 5.0, 4.0, seed=2)
    s = make_system(w, params_for(w))
    for k, v in SETTABLE.items():
        s.set_option(k, v)
        assert s.get_option(k) == v, k
    for k, v in INVALID.items():
        before = s.get_option(k)
        with pytest.raises(dpd.DPDError) as e:
            s.set_option(k, v)
        assert e.value.code == dpd.DPD_EINVAL, k
        assert s.get_option(k) == before, k
    for k in ("ncells", "kernel_launches", "kernels_per_step", "force_variants", "force_newton3",
              "kBT", "dt", "scan_tiles"):
        s.get_option(k)
        with pytest.raises(dpd.DPDError):
            s.set_option(k, 1.0)
    assert s.get_option("ncells") == 6 * 5 * 6
    s.step(2)  # the state still steps with every option changed (graph off, law 1, ...)
    s.close()
