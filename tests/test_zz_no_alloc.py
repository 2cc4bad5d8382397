"""The allocation-free GB energy entry point, cph_gb_energy_noalloc.

Some callers cannot allocate device memory (a plug-in running inside a host
program that owns the whole device-memory budget, or a loop that cannot
afford the device-wide synchronisation of cudaMalloc/cudaFree); this entry
point takes only inputs and output and keeps its scratch in a fixed array
inside the library.  Both entry points run the same kernels with
deterministic int64 fixed-point sums, so the energies must equal those of
cph_gb_energy with a caller workspace bit for bit, on consecutive calls that
reuse the shared array, including a small call right after a large one with
other inputs (nothing left in the array may leak into the next result).  The
calls must not change the device memory in use, and sizes beyond the array
must be refused.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1809_07726_gb300 import build, cphremd, synth

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    f = cphremd.lib().cph_gb_energy_noalloc
    f.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.POINTER(cphremd.GBParams), C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def _inputs(n_rep, n, seed):
    import torch
    s, x, q, rho = synth.config_c5(n_rep=n_rep, n=n, seed=seed)
    dev = "cuda:0"
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    return t(x), t(q), t(rho), t(s.screen)


def _call_noalloc(fn, x, q, rho, screen, E):
    import torch
    n_rep, n = q.shape
    g = cphremd.default_gb()
    st = torch.cuda.current_stream().cuda_stream
    rc = fn(n_rep, n, C.c_void_p(x.data_ptr()), C.c_void_p(q.data_ptr()), C.c_void_p(rho.data_ptr()),
            C.c_void_p(screen.data_ptr()), C.byref(g), C.c_void_p(E.data_ptr()), C.c_void_p(st))
    assert rc == cphremd.OK, cphremd.lib().cph_last_error(None)


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    import torch
    build.build()
    fn = _noalloc_fn()
    # small, larger, the largest that fits (17 x 8000 replica-atoms), then small
    # again with other inputs: every call reuses what the previous one left
    cases = [(71, 6, 700), (72, 3, 1500), (73, 17, 8000), (74, 5, 333)]
    for seed, n_rep, n in cases:
        x, q, rho, scr = _inputs(n_rep, n, seed)
        want = cphremd.gb_energy(x, q, rho, scr).cpu().numpy()
        E = torch.empty(n_rep, dtype=torch.float64, device=q.device)
        _call_noalloc(fn, x, q, rho, scr, E)
        np.testing.assert_array_equal(E.cpu().numpy(), want)


def test_noalloc_calls_allocate_no_device_memory():
    """After one warm-up call per size (which loads the kernels and looks up
    the array's address), further calls change neither the caching
    allocator's count nor the device's free memory."""
    import torch
    build.build()
    fn = _noalloc_fn()
    sets = []
    for seed, n_rep, n in ((81, 4, 900), (82, 2, 2500)):
        x, q, rho, scr = _inputs(n_rep, n, seed)
        E = torch.empty(n_rep, dtype=torch.float64, device=q.device)
        _call_noalloc(fn, x, q, rho, scr, E)
        sets.append((x, q, rho, scr, E))
    torch.cuda.synchronize()
    first = [E.cpu().numpy() for *_, E in sets]
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for (x, q, rho, scr, E) in sets:
            _call_noalloc(fn, x, q, rho, scr, E)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    for want, (*_, E) in zip(first, sets):
        np.testing.assert_array_equal(E.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    fn = _noalloc_fn()
    g = cphremd.default_gb()
    big = 1 << 20  # replica-atoms; needs ~92 MB of scratch (88 B each), the array holds 12 MiB
    rc = fn(16, big // 16, None, None, None, None, C.byref(g), None, None)
    assert rc == cphremd.E_INVALID
    assert b"too large" in cphremd.lib().cph_last_error(None)
    # one replica-atom past the limit is refused too
    lim = 17 * 8000
    while cphremd.gb_workspace_bytes(1, lim + 1) <= (12 << 20):
        lim += 1
    rc = fn(1, lim + 1, None, None, None, None, C.byref(g), None, None)
    assert rc == cphremd.E_INVALID
