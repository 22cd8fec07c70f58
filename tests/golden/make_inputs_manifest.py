"""Write tests/golden/inputs_manifest.json: sha256 digests of the seeded draws
behind every benchmark workload, so that a change of the input recipe (or of
the random stream) is caught by the CPU tests.

For each single-matrix workload the digests cover the drawn spectrum e and the
N(0,1) matrix G whose QR gives the eigenvectors (QR itself is left out: its
last bits depend on the LAPACK build). For the batch the digest covers the
drawn sizes and member seeds. Only `synth` is called; nothing here computes
any step of the method.

    python tests/golden/make_inputs_manifest.py
"""

from __future__ import annotations

import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import CONFIGS, batch_sizes, spectrum  # noqa: E402

MANIFEST = os.path.join(HERE, "inputs_manifest.json")


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float64).tobytes()).hexdigest()


def draws(index: int):
    """(e, G) in the order make_hamiltonian draws them from default_rng(seed)."""
    c = CONFIGS[index]
    rng = np.random.default_rng(c["seed"])
    e = spectrum(c["n"], c["n_occ"], c["occ"], c["virt"], rng)
    G = rng.standard_normal((c["n"], c["n"]))
    return e, G


def manifest() -> dict:
    out = {"numpy": np.__version__, "configs": {}}
    for index in (0, 1, 2, 4):
        e, G = draws(index)
        out["configs"][str(index)] = {"n": int(e.shape[0]), "spectrum_sha256": digest(e), "gaussian_sha256": digest(G)}
    sizes = np.array(batch_sizes(), dtype=np.float64)
    out["configs"]["3"] = {"batch": int(sizes.shape[0]), "sizes_and_seeds_sha256": digest(sizes)}
    return out


if __name__ == "__main__":
    with open(MANIFEST, "w") as f:
        json.dump(manifest(), f, indent=1)
        f.write("\n")
    print(MANIFEST)
