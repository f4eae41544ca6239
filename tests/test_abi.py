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


def test_null_plan_rejected_without_a_device(lib):
    """Every plan entry point checks its arguments before any CUDA call, so a null plan (or
    negative size) is refused with QH_ERR_INVALID_ARG on a machine without a GPU too."""
    import ctypes

    x = (ctypes.c_float * 8)()
    out = (ctypes.c_int32 * 4)()
    cnt = ctypes.c_int32(0)
    p, o, c = ctypes.addressof(x), ctypes.addressof(out), ctypes.byref(cnt)
    assert lib.qh_hull2d_p(None, p, 4, o, c, None) == 1
    assert lib.qh_hull2d_sorted(None, p, 4, o, c, None) == 1
    assert lib.qh_hull2d_host(None, p, 4, o, c, None) == 1
    assert lib.qh_hull2d_batched(None, p, None, 1, o, c, None) == 1
    assert lib.qh_plan_destroy(None) == 0
    assert lib.qh_check_orient_host(p, -1, 0, o, o) == 1


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


def _near_collinear(rng, scale, count):
    """Triples on (or one ulp off) a float line y = fl(0.7 x), coordinates ~scale."""
    out = []
    for _ in range(count):
        x = np.sort(rng.random(3)).astype(np.float32) * np.float32(scale)
        y = (np.float32(0.7) * x).astype(np.float32)
        k = rng.integers(0, 3)
        if k:
            y[1] = np.nextafter(y[1], np.float32((-1) ** k * np.inf))
        out.append([x[0], y[0], x[2], y[2], x[1], y[1]])
    return out


def test_host_exact_paths_across_magnitudes(lib):
    """The exact fallback runs in FP32 for factors in [2^-51, 2^61] (or zero) and
    in FP64 outside; both sides of both limits, mixed scales and zeros agree
    with rational arithmetic."""
    import paper_1501_04706_gb300 as qh

    rng = np.random.default_rng(11)
    tri = []
    for e in [-80, -60, -52, -51, -50, -20, 0, 20, 59, 60, 61, 62, 80]:
        tri += _near_collinear(rng, 2.0 ** e, 150)
        # exactly collinear: small integer multiples of one direction, scaled by 2^e
        for _ in range(20):
            d = rng.integers(-7, 8, size=2)
            k = rng.integers(-9, 10, size=3)
            tri.append([float(np.float32(2.0 ** e) * np.float32(v)) for i in k for v in (i * d[0], i * d[1])])
    # mixed scales inside one triple, and exact zeros
    for _ in range(600):
        t = (rng.random(6) * 2 - 1).astype(np.float32)
        t *= np.float32(2.0) ** rng.integers(-70, 70, size=6).astype(np.float32)
        t[rng.random(6) < 0.2] = 0
        tri.append(list(t))
    tri = np.array(tri, dtype=np.float32)
    assert np.isfinite(tri).all()
    want = np.array([orient(t[0:2], t[2:4], t[4:6]) for t in tri])
    for prec in (0, 1):
        sign, cert = qh.check_orient_host(tri, prec)
        assert np.array_equal(sign, want), prec
    assert (want == 0).sum() > 100  # exact zeros were exercised

    q = []
    for e in [-80, -52, -51, -50, 0, 60, 61, 62, 80]:
        for t in _near_collinear(rng, 2.0 ** e, 120):
            # chord = first two points; p, q = third point and a one-ulp shift of it
            p = np.array(t[4:6], dtype=np.float32)
            qq = p.copy()
            qq[rng.integers(0, 2)] = np.nextafter(qq[0], np.float32(np.inf)) if rng.random() < 0.5 else qq[1]
            q.append(list(t[0:4]) + list(p) + list(qq))
    q = np.array(q, dtype=np.float32)
    got = qh.check_dist_host(q)
    wantd = np.array([dist_sign(t[0:2], t[2:4], t[4:6], t[6:8]) for t in q])
    assert np.array_equal(got, wantd)


def test_host_exact_paths_far_apart_exponents(lib):
    """Nearly and exactly collinear triples on y = x whose coordinates lie up to 2^120
    apart: some differences are exact in FP64 and some are not, so every stage of
    the exact fallback (FP64 difference form, product comparison, expansions) is
    reached; all agree with rational arithmetic."""
    import paper_1501_04706_gb300 as qh

    rng = np.random.default_rng(13)
    tri = []
    for _ in range(600):
        e = rng.integers(-60, 61, size=3).astype(np.float32)
        x = ((np.float32(1.0) + rng.random(3).astype(np.float32)) * np.float32(2.0) ** e).astype(np.float32)
        y = x.copy()
        k = int(rng.integers(0, 3))
        if k:
            y[2] = np.nextafter(y[2], np.float32((-1) ** k * np.inf))
        tri.append([x[0], y[0], x[1], y[1], x[2], y[2]])
    tri = np.array(tri, dtype=np.float32)
    assert np.isfinite(tri).all()
    sign, _ = qh.check_orient_host(tri, 0)
    assert np.array_equal(sign, np.array([orient(t[0:2], t[2:4], t[4:6]) for t in tri]))
    q = np.concatenate([tri, tri[:, 4:6] * np.float32(1.0)], axis=1)
    q[:, 7] = np.nextafter(q[:, 7], np.float32(np.inf))
    got = qh.check_dist_host(q)
    assert np.array_equal(got, np.array([dist_sign(t[0:2], t[2:4], t[4:6], t[6:8]) for t in q]))
