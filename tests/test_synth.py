"""The seeded input generators: reproducible, with the spectra they claim."""

import numpy as np

from synth import CONFIGS, batch_sizes, config_hamiltonian, make_hamiltonian, symmetric_gaussian


def test_seeded_and_reproducible():
    a = make_hamiltonian(50, 10, seed=3)
    b = make_hamiltonian(50, 10, seed=3)
    assert np.array_equal(a.H, b.H) and np.array_equal(a.e, b.e)
    c = make_hamiltonian(50, 10, seed=4)
    assert not np.array_equal(a.H, c.H)


def test_spectrum_and_structure():
    h = config_hamiltonian(0)
    assert h.H.shape == (256, 256) and np.array_equal(h.H, h.H.T)
    assert np.allclose(h.Q.T @ h.Q, np.eye(256), atol=1e-12)
    assert np.all(h.e[:64] <= -0.1) and np.all(h.e[:64] >= -2.0)
    assert np.all(h.e[64:] >= 0.1) and np.all(h.e[64:] <= 2.0)
    w = np.linalg.eigvalsh(h.H)
    assert np.allclose(w, np.sort(h.e), atol=1e-12)


def test_lcao_decay_variant_keeps_spectrum():
    h = make_hamiltonian(128, 32, occ=(-2.0, -0.025), virt=(0.025, 2.0), seed=9, decay=16.0)
    w = np.linalg.eigvalsh(h.H)
    assert np.allclose(w, h.e, atol=1e-12)  # e is sorted for this variant
    assert np.all(h.e[:32] < 0) and np.all(h.e[32:] > 0)


def test_batch_sizes():
    sizes = batch_sizes()
    assert len(sizes) == CONFIGS[3]["batch"]
    for n, n_occ, _ in sizes:
        assert n % 32 == 0 and 128 <= n <= 1536 and n_occ == n // 4
    assert sizes == batch_sizes()


def test_symmetric_gaussian():
    W = symmetric_gaussian(20, 1)
    assert np.array_equal(W, W.T)


def test_inputs_match_the_manifest():
    """The seeded draws behind every benchmark workload hash to the digests in
    tests/golden/inputs_manifest.json (written by make_inputs_manifest.py),
    and those draws are the ones make_hamiltonian uses."""
    import importlib.util
    import json
    import os

    import numpy as np
    import pytest

    from synth import config_hamiltonian

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_inputs_manifest", os.path.join(here, "make_inputs_manifest.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(mk.MANIFEST) as f:
        stored = json.load(f)
    now = mk.manifest()
    if now["configs"] != stored["configs"] and now["numpy"] != stored["numpy"]:
        pytest.skip(f"numpy {now['numpy']} draws differ from the manifest's numpy {stored['numpy']}")
    assert now["configs"] == stored["configs"]
    # the manifest's draw order is make_hamiltonian's
    e, G = mk.draws(0)
    h = config_hamiltonian(0)
    assert np.array_equal(h.e, e)
    Qg, R = np.linalg.qr(G)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    assert np.array_equal(h.Q, Qg * sgn[None, :])
