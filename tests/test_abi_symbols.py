"""The C-ABI library builds, loads without a GPU, and exports every function
declared in include/*.h; the binding declares the same set."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(mem_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libmem():
    from paper_1407_7595_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_all_declared_symbols_exported(libmem):
    names = declared_functions()
    assert {"mem_create_process", "mem_upload_events", "mem_integrate", "mem_destroy"} <= names
    for n in sorted(names):
        assert hasattr(libmem, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header():
    from paper_1407_7595_gb300 import abi
    assert {s[0] for s in abi.SIGNATURES} == declared_functions()


def test_host_only_entry_points(libmem):
    """Calls that need no device: dimension tables and argument validation."""
    from paper_1407_7595_gb300 import abi, synth
    L = abi.lib()
    assert [L.mem_process_dims(k) for k in (0, 1, 2, 3, 4, 5)] == [2, 4, 7, 6, 8, 8]
    assert [L.mem_process_nperm(k) for k in (0, 1, 2, 3, 4, 5)] == [1, 1, 24, 2, 12, 12]
    assert L.mem_process_dims(7) == -1
    d = abi.process_desc(0, synth.DEFAULT_PROCESS)
    d.mz = -1.0
    with pytest.raises(abi.MemError) as e:
        abi.mem_create_process(d)
    assert e.value.status == abi.MEM_ERR_INVALID_ARG
    d = abi.process_desc(9, synth.DEFAULT_PROCESS)       # no such process
    with pytest.raises(abi.MemError):
        abi.mem_create_process(d)
    d = abi.process_desc(4, dict(synth.DEFAULT_PROCESS, wh=0.0))   # ttH needs a Higgs width
    with pytest.raises(abi.MemError):
        abi.mem_create_process(d)
    h = abi.mem_create_process(abi.process_desc(1, synth.DEFAULT_PROCESS))
    abi.mem_destroy(h)
    abi.mem_destroy(None)


def test_ttbb_colour_factors_reproduce_the_oracle_matrices(libmem, ora):
    """The kernels evaluate the colour sums as sum_k |u_k^dagger L|^2 with the library's
    factors K = sum_k u_k u_k^dagger: those factors, rebuilt into a matrix, equal the
    oracle's colour matrices to FP32 rounding (so L^dagger K L is unchanged), and their
    number is the matrices' rank (the oracle's eigenvalues above 1e-10 of the largest:
    11 for g g, 4 for q qbar)."""
    import numpy as np
    from paper_1407_7595_gb300 import abi
    ugg, uqq, ranks = abi.mem_ttbb_colour_factors()
    ogg, oqq = ora.ttbb_colour_matrices()
    for w, o, r in ((ugg, ogg, ranks[0]), (uqq, oqq, ranks[1])):
        ev = np.linalg.eigvalsh(o)
        assert r == int(np.sum(ev > 1e-10 * ev.max()))
        assert np.all(w[r:] == 0)
        u = w[:r].astype(np.complex128).conj()          # rows u_k
        rebuilt = u.T @ u.conj()                        # sum_k u_k u_k^dagger
        scale = np.max(np.abs(o))
        assert np.max(np.abs(rebuilt - o)) < 1e-6 * scale
        rng = np.random.default_rng(3)
        L = rng.normal(size=o.shape[0]) + 1j * rng.normal(size=o.shape[0])
        assert np.sum(np.abs(w[:r].astype(np.complex128) @ L) ** 2) == pytest.approx(
            np.real(L.conj() @ o @ L), rel=1e-5)


def test_ttbb_colour_matrices_match_the_oracle(libmem, ora):
    """The colour matrices the GPU kernels use (computed on the host by the library, with
    its own SU(3) code) equal the oracle's, term by term, to FP32 rounding: the term
    order, the colour tensors and the f^{abc} conventions of the two sides agree."""
    import numpy as np
    from paper_1407_7595_gb300 import abi
    kgg, kqq = abi.mem_ttbb_colour_matrices()
    ogg, oqq = ora.ttbb_colour_matrices()
    for k, o in ((kgg, ogg), (kqq, oqq)):
        scale = np.max(np.abs(o))
        assert scale > 0
        assert np.max(np.abs(k.astype(np.complex128) - o)) < 1e-6 * scale
        assert np.allclose(o, o.conj().T, rtol=0, atol=1e-12 * scale)   # Hermitian
