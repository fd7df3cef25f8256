"""The allocation-free internal-force entry point.

Some callers may not allocate device memory: an application that has frozen its GPU memory budget
and forbids cudaMalloc / cudaFree after start-up, code running inside another allocator's hooks, or
a thread that must never block on cudaFree's implicit synchronisation.  osam_hex8_force_noalloc
serves them from a static device buffer.  Through the C ABI, its result must equal
osam_hex8_force's on two consecutive calls (the buffer is reused), and a mesh beyond the buffer's
limit must be refused with OSAM_EINVAL.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_and_torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_20687_gb300 import build_lib, osam
    build_lib.build()
    return osam, osam.load(), torch


def test_noalloc_force_matches_allocating_entry_point(lib_and_torch):
    osam, L, torch = lib_and_torch
    from paper_2511_20687_gb300 import workloads as W
    lam, mu = W.lame(1e9, 0.25)
    dims, h = (23, 17, 19), 0.01          # 7429 elements, ragged against the 128-thread blocks
    nn = 24 * 18 * 20
    ne = 23 * 17 * 19
    rng = np.random.default_rng(77)
    for call, material in enumerate((osam.NEO_HOOKEAN, osam.LINEAR_ELASTIC)):
        u = torch.tensor(1e-4 * rng.standard_normal((nn, 3)), device="cuda")
        lam_e = torch.tensor(lam * (1 + 0.1 * rng.uniform(-1, 1, ne)), device="cuda") if call else None
        mu_e = torch.tensor(mu * (1 + 0.1 * rng.uniform(-1, 1, ne)), device="cuda") if call else None
        f_ref = torch.empty_like(u)
        f_new = torch.full_like(u, float("nan"))
        args = (dims[0], dims[1], dims[2], h, material, lam, mu,
                None if lam_e is None else lam_e.data_ptr(), None if mu_e is None else mu_e.data_ptr(),
                u.data_ptr())
        assert L.osam_hex8_force(*args, f_ref.data_ptr(), None) == osam.OK
        assert L.osam_hex8_force_noalloc(*args, f_new.data_ptr(), None) == osam.OK
        torch.cuda.synchronize()
        ref = f_ref.cpu().numpy()
        new = f_new.cpu().numpy()
        assert np.all(np.isfinite(new))
        assert np.abs(new - ref).max() < 1e-12 * np.abs(ref).max()


def test_noalloc_force_rejects_meshes_beyond_its_buffer(lib_and_torch):
    osam, L, torch = lib_and_torch
    dims = (64, 32, 17)                    # 34816 elements > OSAM_NOALLOC_MAX_ELEMENTS = 32768
    nn = 65 * 33 * 18
    u = torch.zeros((nn, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros_like(u)
    rc = L.osam_hex8_force_noalloc(dims[0], dims[1], dims[2], 0.01, osam.NEO_HOOKEAN, 1.0, 1.0, None, None,
                                   u.data_ptr(), f.data_ptr(), None)
    assert rc == osam.EINVAL
    msg = L.osam_last_error(None).decode()
    assert "32768" in msg and "34816" in msg
