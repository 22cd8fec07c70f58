"""dm_purify_host: the purification with H and P in host memory, both copies
made inside the library's C ABI. Its result must be the bits of dm_purify on a
device copy of the same H, for pinned and pageable host buffers and for host
leading dimensions larger than n; argument and workspace errors come back as
codes before anything is written."""

import ctypes

import numpy as np
import pytest
import torch

from synth import make_hamiltonian

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,s,refine", [("int8", 7, 0), ("int8", 5, 8), ("e4m3", 7, 0), ("fp64", 0, 0)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_is_bit_identical_to_the_device_call(dmp, mode, s, refine, pinned):
    n, n_occ = 300, 75
    h = make_hamiltonian(n, n_occ, seed=77)
    kw = dict(mode=mode, slices=s, executor="tc" if mode != "fp64" else "auto", tol=1e-10, refine=refine)
    P_dev, info_dev = dmp.purify(torch.from_numpy(h.H).cuda(), n_occ, **kw)
    # host buffers with leading dimensions larger than n (views into wider arrays)
    Hbig = torch.zeros((n, n + 13), dtype=torch.float64, pin_memory=pinned)
    Hbig[:, :n] = torch.from_numpy(h.H)
    Pbig = torch.full((n, n + 7), float("nan"), dtype=torch.float64, pin_memory=pinned)
    H_host, P_host = Hbig[:, :n], Pbig[:, :n]
    opts = dmp.make_opts(mode, s, kw["executor"], 1e-10, refine=refine)
    ws = dmp.workspace(dmp.host_workspace_bytes(n, opts))
    info = dmp.Info()
    rc = dmp.lib().dm_purify_host(H_host.data_ptr(), n, H_host.stride(0), n_occ, ctypes.byref(opts),
                                  P_host.data_ptr(), P_host.stride(0), ctypes.byref(info), ws.data_ptr(),
                                  ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == info_dev["status"] and rc >= 0
    assert torch.equal(P_host, P_dev.cpu())
    assert torch.isnan(Pbig[:, n:]).all()  # nothing written past each row
    assert info.iters == info_dev["iters"] and info.energy == info_dev["energy"]


def test_binding_round_trip(dmp):
    h = make_hamiltonian(256, 64, seed=5)
    H_host = torch.from_numpy(h.H).pin_memory()
    P, info = dmp.purify_host(H_host, 64, mode="int8", slices=7, executor="tc")
    assert not P.is_cuda and P.is_pinned()
    P_dev, info_dev = dmp.purify(torch.from_numpy(h.H).cuda(), 64, mode="int8", slices=7, executor="tc")
    assert torch.equal(P, P_dev.cpu()) and info["status"] == info_dev["status"]


def test_errors_leave_the_output_untouched(dmp):
    n = 128
    h = make_hamiltonian(n, 32, seed=6)
    H_host = torch.from_numpy(h.H)
    P_host = torch.full((n, n), 7.0, dtype=torch.float64)
    opts = dmp.make_opts("int8", 7, "tc")
    need = dmp.host_workspace_bytes(n, opts)
    ws = dmp.workspace(need)
    L = dmp.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    before = dmp.launch_count()
    # n_occ outside (0, n)
    assert L.dm_purify_host(H_host.data_ptr(), n, n, 0, ctypes.byref(opts), P_host.data_ptr(), n, None,
                            ws.data_ptr(), ws.numel(), stream) == dmp.ERR_INVALID_ARG
    # workspace one byte short
    assert L.dm_purify_host(H_host.data_ptr(), n, n, 32, ctypes.byref(opts), P_host.data_ptr(), n, None,
                            ws.data_ptr(), need - 1, stream) == dmp.ERR_WORKSPACE
    # leading dimension below n
    assert L.dm_purify_host(H_host.data_ptr(), n, n - 1, 32, ctypes.byref(opts), P_host.data_ptr(), n, None,
                            ws.data_ptr(), ws.numel(), stream) == dmp.ERR_INVALID_ARG
    assert dmp.launch_count() == before
    assert bool((P_host == 7.0).all())
    # a NaN in H: the error code, and P is not written
    H_bad = H_host.clone()
    H_bad[3, 5] = H_bad[5, 3] = float("nan")
    rc = L.dm_purify_host(H_bad.data_ptr(), n, n, 32, ctypes.byref(opts), P_host.data_ptr(), n, None,
                          ws.data_ptr(), ws.numel(), stream)
    assert rc == dmp.ERR_NONFINITE
    assert bool((P_host == 7.0).all())
