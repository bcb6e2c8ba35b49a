"""Pins for the oracle's random streams (Philox4x32-10, Salmon et al. SC'11).

The generator is checked against an independent implementation, Triton's
``philox_impl``, run on the CPU through Triton's interpreter (a library
routine, executed, not read), and the stream layout is checked for
uniformity and independence of history ids.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats

import oracle

_TRITON_SCRIPT = textwrap.dedent(r"""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl
    from triton.language.random import philox_impl

    @triton.jit
    def k(c_ptr, key_ptr, out_ptr, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c_ptr + 4 * i + 0, mask=m).to(tl.uint32)
        c1 = tl.load(c_ptr + 4 * i + 1, mask=m).to(tl.uint32)
        c2 = tl.load(c_ptr + 4 * i + 2, mask=m).to(tl.uint32)
        c3 = tl.load(c_ptr + 4 * i + 3, mask=m).to(tl.uint32)
        k0 = tl.load(key_ptr + 2 * i + 0, mask=m).to(tl.uint32)
        k1 = tl.load(key_ptr + 2 * i + 1, mask=m).to(tl.uint32)
        o0, o1, o2, o3 = philox_impl(c0, c1, c2, c3, k0, k1)
        tl.store(out_ptr + 4 * i + 0, o0.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 1, o1.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 2, o2.to(tl.int64), mask=m)
        tl.store(out_ptr + 4 * i + 3, o3.to(tl.int64), mask=m)

    data = json.loads(sys.stdin.read())
    c = torch.tensor(data["c"], dtype=torch.int64)
    key = torch.tensor(data["k"], dtype=torch.int64)
    n = c.shape[0]
    out = torch.zeros(n, 4, dtype=torch.int64)
    k[(1,)](c, key, out, n, BLOCK=64)
    print(json.dumps((out & 0xffffffff).tolist()))
""")


def _triton_philox(counters, keys):
    import json
    env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(
        {"c": [[int(v) for v in c] for c in counters], "k": [[int(v) for v in k] for k in keys]}),
        capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip(f"triton interpreter unavailable: {p.stderr.strip()[-200:]}")
    return np.array(json.loads(p.stdout.strip().splitlines()[-1]), dtype=np.uint64)


def test_philox_matches_triton_library_routine():
    pytest.importorskip("triton")
    rng = np.random.default_rng(12345)
    counters = [[0, 0, 0, 0], [0xFFFFFFFF] * 4] + rng.integers(0, 2**32, size=(30, 4)).tolist()
    keys = [[0, 0], [0xFFFFFFFF] * 2] + rng.integers(0, 2**32, size=(30, 2)).tolist()
    want = _triton_philox(counters, keys)
    got = np.array([oracle.philox4x32_10(c, k) for c, k in zip(counters, keys)], dtype=np.uint64)
    np.testing.assert_array_equal(got, want)


def test_stream_layout_blocks_and_histories():
    # history h, block b -> counter (b_lo, b_hi, h_lo, h_hi), key (seed_lo, seed_hi)
    seed, h = 0x0123456789ABCDEF, 0x00000002_80000001
    u = oracle.uniforms(seed, h, 12)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    words = np.concatenate([oracle.philox4x32_10([b, 0, h & 0xFFFFFFFF, h >> 32], key) for b in range(3)])
    np.testing.assert_array_equal(u, (words.astype(np.float64) + 0.5) / 2.0**32)
    assert np.all(u > 0.0) and np.all(u < 1.0)


def test_stream_uniformity_and_independence():
    u = np.concatenate([oracle.uniforms(7, h, 64) for h in range(2000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    a = np.array([oracle.uniforms(7, h, 1)[0] for h in range(4000)])
    b = np.array([oracle.uniforms(7, h + 1, 1)[0] for h in range(4000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 5.0 / np.sqrt(4000)
