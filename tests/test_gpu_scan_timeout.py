"""The single-pass cell scan waits on its predecessors with a bound: a tile that never
publishes (a test hook, option "scan_stall_tile") makes the next tile give up, the
step returns DPD_ETIMEOUT promptly, the kernels that index through the cell starts do
nothing, and the system steps normally again once the state is reloaded.  No GPU
wait is left hanging: the call returns within a few seconds."""
import time

import numpy as np
import pytest

from paper_1807_09896_gb300 import dpd, inputs
from parity_helpers import gpu_state, make_system, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_a_stalled_scan_tile_times_out_and_the_system_recovers(use_graph):
    w = inputs.channel(24.0, 16.0, 14.0, seed=41)  # 24 x 16 x 16 cells: 3 tiles of 2048
    p = params_for(w, g=(0.02, 0.0, 0.0), seed=3)
    s = make_system(w, p, use_graph=use_graph, graph_steps=4)
    ref = make_system(w, p, use_graph=use_graph, graph_steps=4)
    assert s.get_option("scan_tiles") == 3
    s.set_option("scan_stall_tile", 1)
    t0 = time.perf_counter()
    with pytest.raises(dpd.DPDError) as e:
        s.step(4)
    assert e.value.code == dpd.DPD_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # the error is sticky until the state is reloaded
    with pytest.raises(dpd.DPDError) as e:
        s.step(1)
    assert e.value.code == dpd.DPD_ETIMEOUT
    s.set_option("scan_stall_tile", -1)
    s.set_option("step", 0)
    s.set_particles(w.pos4(), w.vel4(), w.id, w.type)
    s.step(6)
    ref.step(6)
    for x, y in zip(gpu_state(s), gpu_state(ref)):
        np.testing.assert_array_equal(x, y)
    s.close()
    ref.close()

