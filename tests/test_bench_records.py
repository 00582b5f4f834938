"""Host-side pieces of the benchmark that need no GPU: the committed DRAM
traffic record is used only for the kernel source it was captured on, and
the float-float arithmetic that the energy reduction uses for FP32/FP16
fields keeps the sums within ~1e-15 of FP64 per-cell terms (checked here on
a NumPy emulation of its FP32 operation sequence)."""
import hashlib
import json
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_matches_the_kernel_source_it_names():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    assert recs, "no traffic record committed"
    for kernel, rec in recs.items():
        src = os.path.join(ROOT, rec["source"])
        assert os.path.exists(src)
        assert rec["dram_bytes_per_launch"] > 0
        assert "--clock-control none" in rec["command"]
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        got = bench.recorded_traffic(kernel, os.path.basename(src), rec.get("grid"))
        # valid only while the source is the captured one
        assert (got == rec["dram_bytes_per_launch"]) == (sha == rec["source_sha256"])


def test_traffic_record_rejects_another_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    csrc = tmp_path / "paper_2105_09671_gb300" / "csrc"
    prof.mkdir()
    csrc.mkdir(parents=True)
    (csrc / "k.cuh").write_text("kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()
    (prof / "traffic.json").write_text(json.dumps(
        {"kern": {"source": "paper_2105_09671_gb300/csrc/k.cuh", "source_sha256": sha,
                  "dram_bytes_per_launch": 1234, "grid": [8, 16]}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("kern", "k.cuh") == 1234
    assert bench.recorded_traffic("kern", "k.cuh", (8, 16)) == 1234
    assert bench.recorded_traffic("kern", "k.cuh", (16, 16)) is None  # another grid
    assert bench.recorded_traffic("other", "k.cuh") is None
    (csrc / "k.cuh").write_text("kernel v2\n")
    assert bench.recorded_traffic("kern", "k.cuh") is None


# ------------------------------------------------ float-float energy terms --
_f = np.float32


def _fma(a, b, c):
    # a * b is exact in FP64 for FP32 a, b; one rounding of the sum to FP64
    # and then to FP32 (a double rounding that can differ from a true FMA
    # only in rare ties, far below what the test measures)
    return _f(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = _f(a + b)
    bb = _f(s - a)
    return s, _f(_f(a - _f(s - bb)) + _f(b - bb))


def _two_prod(a, b):
    p = _f(a * b)
    return p, _fma(a, b, -p)


def _square_ff(h, l):
    sh, sl = _two_prod(h, h)
    return sh, _fma(_f(2.0) * h, l, sl)


def _add_ff(acc, t):
    s, e = _two_sum(acc[0], t[0])
    return s, _f(acc[1] + _f(e + t[1]))


def test_float_float_energy_terms_match_fp64_terms():
    rng = np.random.default_rng(7)
    n, group = 2048, 16
    p = rng.uniform(-1.1, 1.1, n).astype(np.float32)
    p[::7], p[::11] = 1.0, -1.0                    # saturated phases
    p[::13] *= np.float32(1e-4)                    # values near 0
    pn = (p + rng.normal(0.0, 1e-3, n)).astype(np.float32)  # a smooth neighbour
    P, PN = p.astype(np.float64), pn.astype(np.float64)
    bulk_ref = np.sum(0.25 * (P * P - 1.0) ** 2)
    grad_ref = np.sum((PN - P) ** 2)
    vol_ref = np.sum(0.5 * (1.0 + P))
    bulk = grad = psum = 0.0
    for g0 in range(0, n, group):
        b = gr = sp = (_f(0), _f(0))
        for i in range(g0, g0 + group):
            x = p[i]
            p2h, p2l = _two_prod(x, x)
            qh, ql = _two_sum(p2h, _f(-1.0))
            b = _add_ff(b, _square_ff(qh, _f(ql + p2l)))
            sp = _add_ff(sp, (x, _f(0)))
            dh, dl = _two_sum(pn[i], -x)
            gr = _add_ff(gr, _square_ff(dh, dl))
        bulk += 0.25 * (np.float64(b[0]) + np.float64(b[1]))
        grad += np.float64(gr[0]) + np.float64(gr[1])
        psum += np.float64(sp[0]) + np.float64(sp[1])
    vol = 0.5 * n + 0.5 * psum
    assert abs(bulk - bulk_ref) <= 1e-13 * bulk_ref
    assert abs(grad - grad_ref) <= 1e-13 * grad_ref
    assert abs(vol - vol_ref) <= 1e-13 * abs(vol_ref)
    # a plain FP32 evaluation of the same terms is far off: the test can fail
    bulk32 = np.sum((0.25 * (p * p - _f(1.0)) ** 2).astype(np.float64))
    assert abs(bulk32 - bulk_ref) > 1e-10 * bulk_ref
