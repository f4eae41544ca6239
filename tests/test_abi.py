"""The C-ABI library builds, loads without a GPU, exports every declared symbol,
and its host-compiled predicate code agrees with exact rational arithmetic."""
import os
import re

import numpy as np
import pytest

from exact import dist_sign, orient

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_04706_gb300 import build as qb

    qb.build()
    import paper_1501_04706_gb300 as qh

    return qh.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qh.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qh_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.qh_status_string(0) == b"ok"
    assert lib.qh_status_string(2) == b"non-finite input coordinate"
    assert lib.qh_version() >= 10000


def _triples(seed=0, count=3000):
    import pins

    rng = np.random.default_rng(seed)
    tri = [sum(map(list, t), []) for t in pins.adversarial_triples(rng, count)]
    for _ in range(count):
        tri.append(list(rng.integers(-3, 4, size=6).astype(np.float32) / np.float32(2)))
    # near-collinear on a float line
    for _ in range(count):
        x = np.sort(rng.random(3).astype(np.float32) * np.float32(100))
        y = (np.float32(0.7) * x).astype(np.float32)
        y[1] = np.nextafter(y[1], np.float32(rng.choice([-1, 1]) * np.inf))
        tri.append([x[0], y[0], x[2], y[2], x[1], y[1]])
    return np.array(tri, dtype=np.float32)


@pytest.mark.parametrize("prec", [0, 1])
def test_host_orient_filter_never_wrong(lib, prec):
    import paper_1501_04706_gb300 as qh

    tri = _triples()
    sign, cert = qh.check_orient_host(tri, prec)
    want = np.array([orient(t[0:2], t[2:4], t[4:6]) for t in tri])
    assert np.array_equal(sign, want)
    # the filter decides most of the random cases on its own
    assert cert.mean() > 0.3


def test_host_distance_compare(lib):
    import paper_1501_04706_gb300 as qh

    rng = np.random.default_rng(5)
    q = []
    for _ in range(2000):
        q.append(rng.integers(-5, 6, size=8).astype(np.float32))
    for _ in range(1000):
        s = np.float32(2.0 ** int(rng.integers(-10, 20)))
        v = (rng.random(8) * s).astype(np.float32)
        v[6:8] = v[4:6]
        v[7] = np.nextafter(v[7], np.float32(np.inf))
        q.append(v)
    q = np.array(q, dtype=np.float32)
    got = qh.check_dist_host(q)
    want = np.array([dist_sign(t[0:2], t[2:4], t[4:6], t[6:8]) for t in q])
    assert np.array_equal(got, want)


def test_loading_without_library_fails_loudly(tmp_path, monkeypatch):
    import paper_1501_04706_gb300 as qh

    monkeypatch.setattr(qh, "_lib", None)
    monkeypatch.setattr(qh, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        qh.load()
