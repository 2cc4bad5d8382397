"""The allocation-free GB energy entry point, cph_gb_energy_noalloc.

Some callers cannot allocate device memory (a plug-in running inside a host
program that owns the whole device-memory budget, or a loop that cannot
afford the device-wide synchronisation of cudaMalloc/cudaFree); this entry
point takes only inputs and output and keeps its scratch in a fixed array
inside the library.  It must give the same energies as cph_gb_energy with a
caller workspace, on consecutive calls that reuse the shared array, and it
must refuse sizes beyond the array.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_1809_07726_gb300 import build, cphremd, synth

pytestmark = pytest.mark.gpu

ENERGY_REL = 1e-6  # the energy bar of the GPU parity tests


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


def _call_noalloc(fn, x, q, rho, screen):
    import torch
    n_rep, n = q.shape
    E = torch.empty(n_rep, dtype=torch.float64, device=q.device)
    g = cphremd.default_gb()
    st = torch.cuda.current_stream().cuda_stream
    rc = fn(n_rep, n, C.c_void_p(x.data_ptr()), C.c_void_p(q.data_ptr()), C.c_void_p(rho.data_ptr()),
            C.c_void_p(screen.data_ptr()), C.byref(g), C.c_void_p(E.data_ptr()), C.c_void_p(st))
    assert rc == cphremd.OK, cphremd.lib().cph_last_error(None)
    return E.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls():
    build.build()
    fn = _noalloc_fn()
    for seed, (n_rep, n) in ((71, (6, 700)), (72, (3, 1500))):
        x, q, rho, scr = _inputs(n_rep, n, seed)
        want = cphremd.gb_energy(x, q, rho, scr).cpu().numpy()
        got = _call_noalloc(fn, x, q, rho, scr)
        np.testing.assert_allclose(got, want, rtol=ENERGY_REL, atol=0)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    fn = _noalloc_fn()
    g = cphremd.default_gb()
    big = 1 << 20  # replica-atoms; needs ~72 MB of scratch, the array holds 12 MiB
    rc = fn(16, big // 16, None, None, None, None, C.byref(g), None, None)
    assert rc == cphremd.E_INVALID
    assert b"too large" in cphremd.lib().cph_last_error(None)
