"""The allocation-free internal-force entry point.

Some callers may not allocate device memory: an application that has frozen its GPU memory budget
and forbids cudaMalloc / cudaFree after start-up, code running inside another allocator's hooks, or
a thread that must never block on cudaFree's implicit synchronisation.  osam_hex8_force_noalloc
serves them from a static device buffer.  Through the C ABI, its result must equal
osam_hex8_force's on two consecutive calls (the buffer is reused) and the CPU oracle's force, a call
after the device's set-up call must leave the device's free memory unchanged, and a mesh beyond the
buffer's limit must be refused with OSAM_EINVAL.  This file is collected last on purpose.
"""
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


def _call(L, fn, dims, h, material, lam, mu, lam_e, mu_e, u, f):
    return getattr(L, fn)(dims[0], dims[1], dims[2], h, material, lam, mu,
                          None if lam_e is None else lam_e.data_ptr(), None if mu_e is None else mu_e.data_ptr(),
                          u.data_ptr(), f.data_ptr(), None)


def test_noalloc_force_matches_allocating_entry_point_and_oracle(lib_and_torch):
    osam, L, torch = lib_and_torch
    from oracle import oracle as O
    from paper_2511_20687_gb300 import workloads as W
    lam, mu = W.lame(1e9, 0.25)
    dims, h = (23, 17, 19), 0.01          # 7429 elements, ragged against the 128-thread blocks
    nn = 24 * 18 * 20
    ne = 23 * 17 * 19
    rng = np.random.default_rng(77)
    names = {osam.NEO_HOOKEAN: "nh", osam.LINEAR_ELASTIC: "le"}
    for call, material in enumerate((osam.NEO_HOOKEAN, osam.LINEAR_ELASTIC)):
        u_np = 1e-4 * rng.standard_normal((nn, 3))
        le_np = lam * (1 + 0.1 * rng.uniform(-1, 1, ne)) if call else None
        me_np = mu * (1 + 0.1 * rng.uniform(-1, 1, ne)) if call else None
        u = torch.tensor(u_np, device="cuda")
        lam_e = torch.tensor(le_np, device="cuda") if call else None
        mu_e = torch.tensor(me_np, device="cuda") if call else None
        f_ref = torch.empty_like(u)
        f_new = torch.full_like(u, float("nan"))
        assert _call(L, "osam_hex8_force", dims, h, material, lam, mu, lam_e, mu_e, u, f_ref) == osam.OK
        assert _call(L, "osam_hex8_force_noalloc", dims, h, material, lam, mu, lam_e, mu_e, u, f_new) == osam.OK
        torch.cuda.synchronize()
        ref = f_ref.cpu().numpy()
        new = f_new.cpu().numpy()
        assert np.all(np.isfinite(new))
        assert np.abs(new - ref).max() < 1e-12 * np.abs(ref).max()
        orc = O.internal_force(dims, h, (0.0, 0.0, 0.0), names[material], lam, mu, u_np,
                               lam_e=le_np, mu_e=me_np).reshape(-1, 3)
        assert np.abs(new - orc).max() < 1e-12 * np.abs(orc).max()


def test_noalloc_force_leaves_free_device_memory_unchanged(lib_and_torch):
    """After the set-up call, further calls (a different mesh size, another material) take no device
    memory: cudaMemGetInfo's free bytes are the same before and after them."""
    osam, L, torch = lib_and_torch
    lam, mu = 1.6e9, 0.4e9
    meshes = [(1, 1, 1), (9, 7, 11), (32, 32, 32)]
    bufs = []
    for dims in meshes:
        nn = (dims[0] + 1) * (dims[1] + 1) * (dims[2] + 1)
        u = torch.tensor(1e-4 * np.random.default_rng(dims[1]).standard_normal((nn, 3)), device="cuda")
        bufs.append((dims, u, torch.empty_like(u)))
    torch.cuda.synchronize()
    # set-up call on this device (a no-op if an earlier test made it already)
    d0, u0, f0 = bufs[0]
    assert _call(L, "osam_hex8_force_noalloc", d0, 0.01, osam.NEO_HOOKEAN, lam, mu, None, None, u0, f0) == osam.OK
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for material in (osam.SAINT_VENANT_KIRCHHOFF, osam.LINEAR_ELASTIC, osam.NEO_HOOKEAN):
        for dims, u, f in bufs[1:]:
            assert _call(L, "osam_hex8_force_noalloc", dims, 0.01, material, lam, mu, None, None, u, f) == osam.OK
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert torch.isfinite(bufs[-1][2]).all()


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
    # dimensions whose product would overflow 64 bits are refused before the product is formed
    big = 1 << 21
    rc = L.osam_hex8_force_noalloc(big, big, big, 0.01, osam.NEO_HOOKEAN, 1.0, 1.0, None, None,
                                   u.data_ptr(), f.data_ptr(), None)
    assert rc == osam.EINVAL
    assert "dimension" in L.osam_last_error(None).decode()
