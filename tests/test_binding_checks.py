"""The Python binding refuses device buffers the C ABI would misuse (CPU only).

The C entry points take raw pointers and cannot see sizes, so the binding
checks each torch tensor before passing its pointer: a CUDA tensor,
contiguous, of the expected element size and at least the length the call
touches.  Without a GPU, a stand-in object plays the CUDA tensor and real CPU
tensors must be refused before the library is called."""
import pytest
import torch

from paper_1007_3509_gb300 import build
from paper_1007_3509_gb300 import hmcpotts as hm


class FakeCuda:
    """Duck-typed stand-in for a CUDA tensor (what the binding's check reads)."""

    def __init__(self, n, itemsize, contiguous=True):
        self.n, self.itemsize, self.contiguous = n, itemsize, contiguous
        self.is_cuda = True

    def is_contiguous(self):
        return self.contiguous

    def element_size(self):
        return self.itemsize

    def numel(self):
        return self.n

    def data_ptr(self):
        return 0x7F0000001000

    @property
    def dtype(self):
        return f"{self.itemsize}-byte"


def test_device_buffer_check():
    assert hm._dev(None, 10, 4, "x") is None
    assert hm._dev(1234, 10, 4, "x") == 1234  # raw pointer: the caller vouches
    assert hm._dev(FakeCuda(10, 4), 10, 4, "x") == 0x7F0000001000
    assert hm._dev(FakeCuda(11, 4), 10, 4, "x") == 0x7F0000001000
    for t, why in ((FakeCuda(9, 4), "at least 10"), (FakeCuda(10, 8), "4-byte"),
                   (FakeCuda(10, 4, contiguous=False), "contiguous"),
                   (torch.empty(10, dtype=torch.int32), "CUDA")):
        with pytest.raises(hm.HPError) as e:
            hm._dev(t, 10, 4, "x")
        assert e.value.code == hm.HP_ERR_ARG and why in str(e.value)


def test_calls_refuse_host_or_short_buffers():
    build.build()
    lat = hm.Lattice(2, (8, 8), 8, 256, 1, 4, hm.FIELD_GRAIN)
    with pytest.raises(hm.HPError) as e:
        lat.hp_bind(torch.empty(64, dtype=torch.int32))
    assert "hp_bind q" in str(e.value) and e.value.code == hm.HP_ERR_ARG
    with pytest.raises(hm.HPError) as e:
        lat.hp_bind(FakeCuda(63, 4))  # one site short
    assert "at least 64" in str(e.value)
    with pytest.raises(hm.HPError) as e:
        lat.hp_grain_counts(FakeCuda(4, 4))  # counts are int64
    assert "8-byte" in str(e.value)
    with pytest.raises(hm.HPError) as e:
        lat.hp_init_voronoi(hm.ORIENT_SO3, FakeCuda(4, 4))  # needs 4 G floats
    assert "at least 16" in str(e.value)
    with pytest.raises(hm.HPError) as e:  # SO(3) texture: bins 2G, histogram 24
        hm.hp_texture(4, hm.ORIENT_SO3, FakeCuda(16, 4), FakeCuda(4, 8), FakeCuda(4, 4), FakeCuda(24, 8))
    assert "bins" in str(e.value) and "at least 8" in str(e.value)
    with pytest.raises(hm.HPError) as e:
        hm.hp_cp_reset(hm.cp_params(250.8e3, 150.0e3, 123.5e3, 60.0, 90.0, 300.0, 1000.0, 1e-4), 10,
                       FakeCuda(59, 4), FakeCuda(10, 4), FakeCuda(10, 4))
    assert "eps_p" in str(e.value) and "at least 60" in str(e.value)
    with pytest.raises(hm.HPError) as e:
        hm.hp_sur_field(FakeCuda(hm.hp_mlp_param_count(), 4), FakeCuda(16, 4), 4, [0.0] * 6, 7.0, FakeCuda(4, 4))
    assert "7 values" in str(e.value)
    lat.close()
