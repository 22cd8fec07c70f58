"""The C-ABI library: it builds, loads without a GPU and exports exactly what
include/dmp.h declares. No compute call is made here."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dmp.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def built():
    from paper_2407_13299_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dm_purify", "ozaki_gemm", "dm_purify_batched", "dm_purify_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_binding_covers_the_header(built):
    from paper_2407_13299_gb300 import dmp

    assert sorted(dmp.SIGNATURES) == _declared_functions()
    L = dmp.lib()
    assert L.dmp_version().decode().startswith("dmp")
    assert dmp.status_str(-5) == "DMP_ERR_UNSUPPORTED"


def test_struct_layouts_match_header(built, tmp_path):
    """Every field offset and the size of each struct of the ABI, as a C compiler
    lays them out from include/dmp.h, equal the binding's ctypes layout."""
    from paper_2407_13299_gb300 import dmp

    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dmp.h"', "int main(void) {"]
    structs = (("dmp_opts", dmp.Opts), ("dmp_info", dmp.Info), ("dmp_foe_params", dmp.FoeParams),
               ("dmp_foe_info", dmp.FoeInfo))
    for cname, cls in structs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                            check=True).stdout.splitlines())
    for cname, cls in structs:
        assert int(got[f"{cname} size"]) == ctypes.sizeof(cls)
        for field, _ in cls._fields_:
            assert int(got[f"{cname} {field}"]) == getattr(cls, field).offset, (cname, field)


def test_workspace_sizes_are_host_side(built):
    from paper_2407_13299_gb300 import dmp

    o = dmp.make_opts("int8", 7, "imma")
    small = dmp.purify_workspace_bytes(256, o)
    big = dmp.purify_workspace_bytes(8192, o)
    # two FP64 n x n buffers + two int8 digit stacks dominate
    assert big >= 2 * 8192 * 8192 * 8 + 2 * 7 * 8192 * 8192
    assert small < big
    f = dmp.purify_workspace_bytes(256, dmp.make_opts("fp64"))
    assert f < small
    assert dmp.tape_bytes(1024, dmp.make_opts("fp64", max_iter=100, checkpoint_every=8)) >= 13 * 1024 * 1024 * 8


# Largest square size ozaki_gemm_noalloc accepts at s = 7, as include/dmp.h states
# it: (mode, executor) -> size (a multiple of 32).
NOALLOC_LIMITS_S7 = {("int8", "tc"): 1056, ("bf16", "tc"): 1056, ("e4m3", "tc"): 1440, ("int8", "imma"): 2432}


@pytest.mark.parametrize("mode,executor", sorted(NOALLOC_LIMITS_S7))
def test_noalloc_limits_in_the_header_hold(built, mode, executor):
    """The sizes the header promises for ozaki_gemm_noalloc fit its 128 MiB array
    and the next multiple of 32 does not, so the documented limit cannot drift
    away from the workspace the product really needs."""
    from paper_2407_13299_gb300 import dmp

    text = open(HEADER).read()
    limit = NOALLOC_LIMITS_S7[(mode, executor)]
    assert str(limit) in text
    cap = 128 << 20
    assert dmp.gemm_workspace_bytes(limit, limit, limit, mode, 7, executor) <= cap
    assert dmp.gemm_workspace_bytes(limit + 32, limit + 32, limit + 32, mode, 7, executor) > cap


def test_argument_errors_without_gpu(built):
    from paper_2407_13299_gb300 import dmp

    L = dmp.lib()
    b = ctypes.c_size_t(0)
    bad = dmp.make_opts("int8", 11, "imma")  # s out of range for beta 7
    assert L.dmp_workspace_size(256, ctypes.byref(bad), ctypes.byref(b)) == dmp.ERR_INVALID_ARG
    assert L.dmp_workspace_size(1, ctypes.byref(dmp.make_opts()), ctypes.byref(b)) == dmp.ERR_INVALID_ARG
    o = dmp.make_opts()
    info = dmp.Info()
    rc = L.dm_purify(None, 16, 16, 4, ctypes.byref(o), None, 16, ctypes.byref(info), None, 0, None, 0, None)
    assert rc == dmp.ERR_INVALID_ARG


def test_option_validation_needs_no_gpu(built):
    """Argument checks of the workspace queries (host-side only): slice ranges
    per mode, executor and method restrictions, and the digit bytes per mode."""
    import ctypes as ct

    from paper_2407_13299_gb300 import dmp

    def ws(n, **kw):
        b = ct.c_size_t(0)
        return dmp.lib().dmp_workspace_size(n, ct.byref(dmp.make_opts(**kw)), ct.byref(b)), b.value

    assert ws(512, mode="e4m3", slices=12, executor="tc")[0] == dmp.OK
    assert ws(512, mode="e4m3", slices=13, executor="tc")[0] == dmp.ERR_INVALID_ARG
    assert ws(512, mode="bf16", slices=10, executor="tc")[0] == dmp.ERR_INVALID_ARG
    assert ws(512, mode="bf16", slices=4, executor="imma")[0] == dmp.ERR_UNSUPPORTED
    assert ws(512, mode="e4m3", slices=4, executor="imma")[0] == dmp.ERR_UNSUPPORTED
    assert ws(512, mode="int8", slices=5, late_slices=4, late_idem=1.0, method="trs4")[0] == dmp.ERR_UNSUPPORTED
    assert ws(512, mode="int8", slices=5, late_slices=11, late_idem=1.0)[0] == dmp.ERR_INVALID_ARG
    # one byte per E4M3 digit against two per bf16-carried digit: the E4M3
    # workspace is the smaller one at equal s
    _, b_e4 = ws(2048, mode="e4m3", slices=8, executor="tc")
    _, b_i8 = ws(2048, mode="int8", slices=8, executor="tc")
    assert b_e4 < b_i8
    n = (ct.c_int64 * 2)(256, 384)
    b = ct.c_size_t(0)
    assert dmp.lib().dmp_batched_workspace_size(2, n, ct.byref(dmp.make_opts("fp64")), ct.byref(b)) == \
        dmp.ERR_UNSUPPORTED
    assert dmp.lib().dmp_batched_workspace_size(2, n, ct.byref(dmp.make_opts("e4m3", 8, "tc")), ct.byref(b)) == \
        dmp.OK


def test_foe_validation_needs_no_gpu(built):
    """dm_foe's argument and option checks run on the host before any CUDA
    call (the device pointers below are never dereferenced)."""
    import ctypes as ct

    from paper_2407_13299_gb300 import dmp

    L = dmp.lib()
    b = ct.c_size_t(0)
    fp = dmp.foe_params(0.05, 64, mu=0.0)
    for kw, want in ((dict(mode="int8", slices=5), dmp.OK), (dict(mode="fp64"), dmp.OK),
                     (dict(mode="e4m3", slices=8, executor="tc"), dmp.OK),
                     (dict(mode="int8", slices=5, refine=7), dmp.ERR_UNSUPPORTED),
                     (dict(mode="int8", slices=5, method="sp2"), dmp.ERR_UNSUPPORTED),
                     (dict(mode="int8", slices=5, fp32_storage=True), dmp.ERR_UNSUPPORTED),
                     (dict(mode="int8", slices=5, late_slices=4, late_idem=1e-3), dmp.ERR_UNSUPPORTED)):
        assert L.dm_foe_workspace_size(512, ct.byref(fp), ct.byref(dmp.make_opts(**kw)), ct.byref(b)) == want, kw
    o = dmp.make_opts("int8", 5)
    assert L.dm_foe_workspace_size(1024, ct.byref(fp), ct.byref(o), ct.byref(b)) == dmp.OK
    assert b.value >= 4 * 1024 * 1024 * 8  # H_s, two recurrence terms and the product
    need = b.value
    # the Paterson-Stockmeyer scheme keeps q = ceil(sqrt(M)) baby steps: 8 for M = 64
    ps = dmp.foe_params(0.05, 64, mu=0.0, scheme="ps")
    assert L.dm_foe_workspace_size(1024, ct.byref(ps), ct.byref(o), ct.byref(b)) == dmp.OK
    assert b.value >= need + 7 * 1024 * 1024 * 8 - 1024 * 1024 * 8
    bad = dmp.foe_params(0.05, 64, mu=0.0)
    bad.scheme = 2
    assert L.dm_foe_workspace_size(1024, ct.byref(bad), ct.byref(o), ct.byref(b)) == dmp.ERR_INVALID_ARG
    bad = dmp.foe_params(0.05, dmp.FOE_MAX_TERMS + 1, mu=0.0)
    assert L.dm_foe_workspace_size(1024, ct.byref(bad), ct.byref(o), ct.byref(b)) == dmp.ERR_INVALID_ARG

    def call(n=1024, ws_bytes=None, **kw):
        p = dict(kT=0.05, mu=0.0, n_occ=0, n_terms=64, scheme=0, e_min=0.0, e_max=0.0)
        p.update(kw)
        params = dmp.FoeParams(**p)
        info = dmp.FoeInfo()
        fake = 1 << 40  # never dereferenced: every case below fails its checks first
        return L.dm_foe(fake, n, n, ct.byref(params), ct.byref(o), fake, n, ct.byref(info), fake,
                        need if ws_bytes is None else ws_bytes, None)

    assert L.dm_foe(None, 16, 16, None, ct.byref(o), None, 16, None, None, 0, None) == dmp.ERR_INVALID_ARG
    assert call(kT=0.0) == dmp.ERR_INVALID_ARG
    assert call(kT=float("inf")) == dmp.ERR_INVALID_ARG
    assert call(mu=float("nan")) == dmp.ERR_INVALID_ARG
    assert call(n_terms=1) == dmp.ERR_INVALID_ARG
    assert call(n_terms=dmp.FOE_MAX_TERMS + 1) == dmp.ERR_INVALID_ARG
    assert call(n_occ=1024) == dmp.ERR_INVALID_ARG
    assert call(n_occ=-1) == dmp.ERR_INVALID_ARG
    assert call(e_min=float("nan")) == dmp.ERR_INVALID_ARG
    assert call(scheme=2) == dmp.ERR_INVALID_ARG
    assert call(n=1) == dmp.ERR_INVALID_ARG
    assert call(ws_bytes=need - 1) == dmp.ERR_WORKSPACE
    assert call(scheme=1) == dmp.ERR_WORKSPACE  # the scheme needs its baby-step slots
    assert call(n=200000) == dmp.ERR_UNSUPPORTED  # level sums of k = n would overflow int32


def test_foe_scheme_slots_need_no_gpu(built):
    """The Paterson-Stockmeyer workspace holds q = ceil(sqrt(M)) baby-step
    slots of n x n doubles (H_s being the first) on top of the recurrence's
    buffers less its separate H_s, plus one more set of digit planes (y = T_q)."""
    import ctypes as ct
    import math

    from paper_2407_13299_gb300 import dmp

    L = dmp.lib()
    n = 512
    nn = n * n * 8
    for mode, slices in (("fp64", 0), ("int8", 5)):
        o = dmp.make_opts(mode, max(slices, 1))
        b_rec, b_ps = ct.c_size_t(0), ct.c_size_t(0)
        for M in (2, 3, 4, 5, 17, 200, 1000, dmp.FOE_MAX_TERMS):
            rec = dmp.foe_params(0.1, M, mu=0.0)
            ps = dmp.foe_params(0.1, M, mu=0.0, scheme="ps")
            assert L.dm_foe_workspace_size(n, ct.byref(rec), ct.byref(o), ct.byref(b_rec)) == dmp.OK
            assert L.dm_foe_workspace_size(n, ct.byref(ps), ct.byref(o), ct.byref(b_ps)) == dmp.OK
            q = math.isqrt(M - 1) + 1 if M > 1 else 1
            extra = b_ps.value - b_rec.value - (q - 1) * nn
            # the third plane set: s planes of n x n bfloat16 digits (n = 512 is
            # already a multiple of the row and K padding) and n int32 exponents;
            # none in FP64 mode
            planes = 0 if mode == "fp64" else slices * n * n * 2 + n * 4
            assert extra == planes, (mode, M, extra)


def test_no_fallback_without_the_library(tmp_path, monkeypatch):
    """Without the compiled library every call fails loudly; nothing falls back
    to a host implementation."""
    import numpy as np
    import torch

    from paper_2407_13299_gb300 import dmp

    monkeypatch.setattr(dmp, "LIB_PATH", str(tmp_path / "missing" / "libdmp.so"))
    monkeypatch.setattr(dmp, "_lib", None)
    with pytest.raises(ImportError):
        dmp.lib()
    with pytest.raises((ImportError, TypeError)):
        dmp.ozaki_gemm(torch.from_numpy(np.eye(4)), torch.from_numpy(np.eye(4)), "int8", 3)
    with pytest.raises(ImportError):
        dmp.purify_workspace_bytes(64, dmp.make_opts("int8", 5))
