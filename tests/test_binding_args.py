"""The Python binding checks every tensor it hands to the C ABI before the call: a host tensor,
a wrong dtype or a short buffer would otherwise reach a kernel as a bad address.  These checks
run on the host, so they are tested here without a GPU (a CPU tensor that passes every other
check is refused for not being on the device)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_15209_gb300 import zeta as Z  # noqa: E402


def test_none_passes_through():
    assert Z._arg(None, "x", torch.float32) is None


def test_rejects_non_tensors():
    with pytest.raises(TypeError, match="particles"):
        Z._f32(np.zeros((4, 4), np.float32), "particles", cols=4)


def test_rejects_wrong_dtype():
    with pytest.raises(ValueError, match="dtype"):
        Z._f32(torch.zeros((4, 4), dtype=torch.float64), "particles", cols=4)
    with pytest.raises(ValueError, match="dtype"):
        Z._f64(torch.zeros(9, dtype=torch.float32), "gram", 9)
    with pytest.raises(ValueError, match="dtype"):
        Z._arg(torch.zeros(9, dtype=torch.int32), "tile_start", torch.int64, 9)


def test_rejects_wrong_particle_layout():
    with pytest.raises(ValueError, match=r"\(N, 4\)"):
        Z._f32(torch.zeros((10, 3)), "particles", cols=4)
    with pytest.raises(ValueError, match=r"\(N, 4\)"):
        Z._f32(torch.zeros(40), "particles", cols=4)


def test_rejects_short_buffers():
    with pytest.raises(ValueError, match="at least 4096"):
        Z._f32(torch.zeros((16, 16, 15)), "delta", 16 ** 3)


def test_rejects_non_contiguous():
    t = torch.zeros((8, 8))[:, ::2]
    with pytest.raises(ValueError, match="contiguous"):
        Z._f32(t, "delta", 16)


def test_refuses_host_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        Z._f32(torch.zeros((10, 4)), "particles", cols=4)
    with pytest.raises(ValueError, match="CUDA"):
        Z._f64(torch.zeros(25, dtype=torch.float64), "gram", 25)
