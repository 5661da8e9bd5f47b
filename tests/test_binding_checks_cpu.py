"""The binding's checks of device buffers, on the CPU.

The C calls that take device arrays (state in/out, halo strips, signal-speed
keys, the network's inputs and outputs, the block average) receive a bare
pointer and cannot see the buffer's size, so the binding refuses a tensor of the
wrong element count, dtype, layout or device before the call.  These tests build
the binding objects without a context, replace the library by a recorder, and
check that a bad buffer raises ValueError without reaching it and a good one
reaches it with its own address.
"""
import ctypes
import types

import numpy as np
import pytest
import torch

from paper_1710_06423_b300 import sac


class FakeDev:
    """A stand-in for a CUDA tensor (no GPU here): what the checks look at."""

    def __init__(self, shape, dtype=torch.float32, contiguous=True, cuda=True, index=0, ptr=0x7000_0000):
        self.shape, self.dtype = tuple(shape), dtype
        self._contig, self.is_cuda, self._ptr = contiguous, cuda, ptr
        self.device = types.SimpleNamespace(index=index if cuda else None, type="cuda" if cuda else "cpu")

    def numel(self):
        return int(np.prod(self.shape))

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return self._ptr


class Recorder:
    """Replaces the loaded library: every call is recorded and returns SAC_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append((name, args))
            if name == "sac_halo_size":
                args[2]._obj.value = 6 * 3 * 22
            return sac.SAC_OK
        return fn


@pytest.fixture
def rec(monkeypatch):
    r = Recorder()
    monkeypatch.setattr(sac, "load", lambda: r)
    return r


def solver(fp32=True, nx=16, ny=16, device=0):
    s = object.__new__(sac.Solver)
    s.nx, s.ny, s.fp32 = nx, ny, fp32
    s.params = types.SimpleNamespace(device=device)
    s._ctx = ctypes.c_void_p(0x1234)
    return s


def cnn(nx=24, ny=16, device=0):
    c = object.__new__(sac.CNN)
    c.nx, c.ny, c.device, c.nparams = nx, ny, device, 4
    c._c = ctypes.c_void_p(0x5678)
    return c


BAD_STATE = [
    FakeDev((6, 16, 15)),                       # too few elements
    FakeDev((6, 16, 16), dtype=torch.float64),  # FP64 into an FP32 context
    FakeDev((6, 16, 16), contiguous=False),
    FakeDev((6, 16, 16), cuda=False),
    FakeDev((6, 16, 16), index=1),              # another GPU
]


@pytest.mark.parametrize("bad", BAD_STATE)
def test_state_buffers_are_refused_before_the_call(rec, bad):
    s = solver()
    with pytest.raises(ValueError):
        s.set_state_dev(bad)
    with pytest.raises(ValueError):
        s.get_state_dev(bad)
    with pytest.raises(ValueError):
        s.set_state_dev(FakeDev((6, 16, 16)), FakeDev((3, 16, 16)))   # background of 3 fields
    assert rec.calls == []


def test_state_buffers_of_the_context_dtype_reach_the_call(rec):
    s = solver(fp32=False, nx=8, ny=4)
    w, bg = FakeDev((6, 4, 8), dtype=torch.float64, ptr=0xA000), FakeDev((4, 4, 8), dtype=torch.float64, ptr=0xB000)
    s.set_state_dev(w, bg, 0.5)
    s.get_state_dev(FakeDev((6 * 4 * 8,), dtype=torch.float64, ptr=0xC000))   # any shape of the right size
    (n1, a1), (n2, a2) = rec.calls
    assert n1 == "sac_set_state_dev" and a1[1].value == 0xA000 and a1[2].value == 0xB000 and a1[3] == 0.5
    assert n2 == "sac_get_state_dev" and a2[1].value == 0xC000
    with pytest.raises(ValueError):
        s.get_state_dev(FakeDev((6, 4, 8), dtype=torch.float32))


def test_halo_strips_and_keys_are_checked(rec):
    s = solver(nx=16, ny=16)
    n = 6 * 3 * 22
    with pytest.raises(ValueError):
        s.halo_pack(0, FakeDev((n - 1,)))
    with pytest.raises(ValueError):
        s.halo_unpack(0, FakeDev((n,), dtype=torch.float64))
    with pytest.raises(ValueError):
        s.get_cmax_bits(FakeDev((2,), dtype=torch.int32))
    with pytest.raises(ValueError):
        s.set_cmax_bits(FakeDev((3,), dtype=torch.int64))
    assert [c[0] for c in rec.calls] == ["sac_halo_size", "sac_halo_size"]
    s.halo_pack(0, FakeDev((n,), ptr=0xD000))
    s.get_cmax_bits(FakeDev((2,), dtype=torch.int64, ptr=0xE000))
    assert rec.calls[-2][0] == "sac_halo_pack" and rec.calls[-2][1][2].value == 0xD000
    assert rec.calls[-1][0] == "sac_get_cmax_bits" and rec.calls[-1][1][1].value == 0xE000


def test_network_buffers_are_checked(rec):
    c = cnn(nx=24, ny=16)
    w, nxt = FakeDev((6, 16, 24), ptr=0x1000), FakeDev((6, 16, 24), ptr=0x2000)
    with pytest.raises(ValueError):
        c.forward(w, 5 / 3, 1 / 24, 1 / 16, FakeDev((16 * 24, 6)))          # pred holds 8 channels
    with pytest.raises(ValueError):
        c.train_step(w, FakeDev((6, 16, 23)), 5 / 3, 1 / 24, 1 / 16, 1e-3)
    with pytest.raises(ValueError):
        c.grads(FakeDev((6, 16, 24), dtype=torch.bfloat16), nxt, 5 / 3, 1 / 24, 1 / 16)
    with pytest.raises(ValueError):
        c.perturb(w, FakeDev((6, 16, 24), index=2), np.ones(6), 1)
    assert rec.calls == []
    c.forward(w, 5 / 3, 1 / 24, 1 / 16, FakeDev((16 * 24, 8), ptr=0x3000))
    name, args = rec.calls[-1]
    assert name == "sac_cnn_forward" and args[1].value == 0x1000 and args[5].value == 0x3000


def test_block_average_sizes_are_checked(rec, monkeypatch):
    monkeypatch.setattr(sac, "_stream_handle", lambda stream, device=0: None)
    fine = FakeDev((6, 32, 48), ptr=0x4000)
    with pytest.raises(ValueError):
        sac.block_average(fine, 6, 48, 32, 5, FakeDev((6, 6, 9)))            # 5 divides neither side
    with pytest.raises(ValueError):
        sac.block_average(fine, 6, 48, 32, 4, FakeDev((6, 8, 11)))
    with pytest.raises(ValueError):
        sac.block_average(fine, 6, 48, 32, 4, FakeDev((6, 8, 12), index=1))  # not with the input
    assert rec.calls == []
    sac.block_average(fine, 6, 48, 32, 4, FakeDev((6, 8, 12), ptr=0x5000))
    name, args = rec.calls[-1]
    assert name == "sac_block_average" and args[0].value == 0x4000 and args[5].value == 0x5000
