"""Handle configuration through the C ABI without a GPU: the defaults, and that
lasto_poisson_create rejects a bad configuration before it touches the device."""
import ctypes

import pytest


def _lib():
    from paper_0806_1723_gb300 import binding
    return binding, binding.load()


def test_defaults():
    binding, _ = _lib()
    cfg = binding.lasto_config_default()
    assert (cfg.n_max, cfg.max_atoms, cfg.max_batch) == (129, 561, 1)
    assert (cfg.nu1, cfg.nu2, cfg.nu_coarse) == (4, 4, 4)
    assert cfg.rel_tol == 1e-10 and cfg.max_cycles == 50
    assert ctypes.sizeof(binding.lasto_config) == ctypes.sizeof(cfg)


@pytest.mark.parametrize("field,value", [("nu_coarse", -1), ("nu_coarse", 65), ("nu1", -1), ("n_max", 64),
                                         ("max_batch", 0), ("rel_tol", 0.0), ("launch", 3), ("boundary", 7),
                                         ("precision", 5), ("n_theta", 33)])
def test_create_rejects_bad_config(field, value):
    binding, L = _lib()
    cfg = binding.lasto_config_default()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert L.lasto_poisson_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.LASTO_ERR_INVALID_ARG
    assert not h.value
