"""Shared helpers of the GPU parity tests (inputs only; no method arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0806_1723_gb300 import binding
    binding.load()
    return binding


def graded_axis(n, L, ratio, seed=0, jitter=0.0):
    """A strictly increasing axis on [-L, L] whose spacing grows smoothly by `ratio` from the centre
    to the edges (test-local recipe, independent of both implementations' mesh builders)."""
    m = (n - 1) // 2
    w = 1.0 + (ratio - 1.0) * (np.abs(np.arange(n - 1) - (n - 2) / 2.0) / ((n - 2) / 2.0)) ** 2
    if jitter:
        w *= 1.0 + jitter * np.random.default_rng(seed).uniform(-1, 1, n - 1)
    x = np.concatenate([[0.0], np.cumsum(w)])
    x = (x / x[-1]) * 2 * L - L
    x[m] = x[m]  # keep as computed
    return x


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()
