"""File checkpoints (dh_save / dh_load): a loaded context continues bit for bit."""
import numpy as np
import pytest
import torch

from paper_2512_13403_b300 import _lib, inputs
from tests.gpu_util import solver, to_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_save_load_continues_bitwise(tmp_path, prec):
    shape = (16, 16, 16)
    kw = dict(forcing=True, cooling=True, gravity=True)
    state = inputs.self_gravitating_box(shape, seed=5, sigma=0.5)
    a = solver(shape, prec, **kw)
    a.init_state(to_gpu(state, prec))
    a.advance(3)
    path = tmp_path / "ck.bin"
    a.save(str(path))
    a.advance(4)
    ref = a.get_state().cpu()
    t_ref = a.time()

    b = solver(shape, prec, **kw)
    b.init_state(to_gpu(inputs.uniform_state(shape), prec))   # overwritten by the load
    b.advance(1)
    b.load(str(path))
    b.advance(4)
    assert torch.equal(b.get_state().cpu(), ref)
    assert b.time() == t_ref
    assert np.array_equal(b.forcing_modes(), a.forcing_modes())


def test_load_rejects_other_configuration_and_corruption(tmp_path):
    shape = (16, 16, 16)
    a = solver(shape, "f32", forcing=True)
    a.init_state(to_gpu(inputs.cooling_box(shape), "f32"))
    a.advance(2)
    path = tmp_path / "ck.bin"
    a.save(str(path))
    other = solver(shape, "f32", forcing=False)
    other.init_state(to_gpu(inputs.cooling_box(shape), "f32"))
    with pytest.raises(_lib.DhError):
        other.load(str(path))
    raw = bytearray(path.read_bytes())
    raw[200] ^= 0xFF
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    b = solver(shape, "f32", forcing=True)
    b.init_state(to_gpu(inputs.cooling_box(shape), "f32"))
    with pytest.raises(_lib.DhError):
        b.load(str(bad))
    with pytest.raises(_lib.DhError):
        b.load(str(tmp_path / "missing.bin"))


@pytest.mark.parametrize("change", [dict(integrator="ssprk3"), dict(limiter="vanleer"), dict(cfl=0.3),
                                    dict(t_floor=0.1), dict(ou_tau=0.4)])
def test_load_rejects_other_scheme_and_settings(tmp_path, change):
    """A checkpoint carries every setting a step depends on: a context with another integrator,
    limiter, CFL number or source setting refuses it (its continuation would not be the saved
    run's), and keeps its own state."""
    shape = (16, 16, 16)
    kw = dict(forcing=True, cooling=True)
    a = solver(shape, "f32", **kw)
    a.init_state(to_gpu(inputs.cooling_box(shape), "f32"))
    a.advance(2)
    path = tmp_path / "ck.bin"
    a.save(str(path))
    b = solver(shape, "f32", **{**kw, **change})
    U = to_gpu(inputs.cooling_box(shape), "f32")
    b.init_state(U)
    with pytest.raises(_lib.DhError) as e:
        b.load(str(path))
    assert e.value.status == _lib.DH_ERR_ARG
    assert "differs" in str(e.value)
    assert torch.equal(b.get_state(), U)
