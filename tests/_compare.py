"""Helpers shared by the GPU parity tests: run the oracle and the CUDA path on
the same seeded inputs and compare what is unique bit for bit."""
import numpy as np

import oracle
from oracle import Scheme as OScheme, Target as OTarget


def oracle_scheme(pscheme, ndim):
    """Oracle scheme equal to a binding Scheme (2-D user axes -> internal 1, 2)."""
    order = pscheme.order
    if order is not None and ndim == 2:
        order = tuple(a + 1 for a in order)
    dax = pscheme.decomp_axis
    return OScheme(mode=pscheme.mode, interp=pscheme.interp, degree=pscheme.degree, order=order,
                   decomp_axis=dax, encoding=pscheme.encoding, nlevels=pscheme.nlevels,
                   nplanes=pscheme.nplanes)


def sign_slot(enc, g):
    """Oracle sign words of segment g laid out as the library's sign slot."""
    words = [w for w in enc["signs"][g]]
    return np.concatenate(words) if words else np.zeros(0, np.uint32)


def compare_streams(h_gpu, h_or, check_pairs=True):
    """Planes, sign areas, sign counts, pair counts and tables of every stream."""
    assert h_gpu.nstreams == len(h_or["streams"])
    for i, s in enumerate(h_or["streams"]):
        info = h_gpu.stream_info(i)
        assert info["n_pad"] == s["n_pad"] and info["n_real"] == s["n_real"], i
        planes, signs, scnt, pairs = h_gpu.stream_copy(i)
        enc = s["enc"]
        assert np.array_equal(planes, enc["planes"]), f"stream {i} planes differ"
        if "sign_counts" in enc:
            assert np.array_equal(scnt.astype(np.int64), enc["sign_counts"]), f"stream {i} sign counts"
            for g in range(scnt.shape[0]):
                want = sign_slot(enc, g)
                assert np.array_equal(signs[g, :want.size], want), f"stream {i} segment {g} signs"
        if check_pairs and "pairs" in enc:
            C = enc["pairs"]
            B = C.shape[0]
            for a in range(B):
                for b in range(a, B):
                    assert int(pairs[a, b]) == int(C[a, b]), (i, a, b)
        tab = h_gpu.tables(i)
        t = s["tab"]
        assert tab["bytes"] == list(t["bytes"]), f"stream {i} bytes"
        assert tab["maxerr"] == list(t["maxerr"]), f"stream {i} maxerr"
        assert tab["sq"] == list(t["sq"]), f"stream {i} sq"


def psnr(x, y, R):
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(y, np.float64)) ** 2))
    return float("inf") if mse == 0 else 20 * np.log10(R / np.sqrt(mse))
