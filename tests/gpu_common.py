"""Shared helpers of the GPU parity tests (imported by tests marked gpu)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08804_gb300 import build
    build.build()


def dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda().contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def logdiff(a, b):
    """|a - b| for complex logs compared mod 2 pi i."""
    d = np.asarray(a) - np.asarray(b)
    im = (d.imag + np.pi) % (2 * np.pi) - np.pi
    return np.abs(d.real + 1j * im)


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
