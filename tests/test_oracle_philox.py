"""Pins for the oracle's Philox4x32-10 (Sec. 4, counter-based generators).

The Random123 known-answer file is not available on these machines, so the
oracle's generator is compared word for word with an independent
Philox4x32-10 that is: PyTorch's header-only CPU engine
(ATen/core/PhiloxRNGEngine.h), compiled here into a small harness. That engine
takes key = seed and counter = (offset lo, offset hi, subsequence lo,
subsequence hi), which maps onto any (counter, key) pair.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned long long n;
  if (scanf("%llu", &n) != 1) return 1;
  for (unsigned long long i = 0; i < n; ++i) {
    unsigned c0, c1, c2, c3, k0, k1;
    if (scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) != 6) return 2;
    uint64_t seed = ((uint64_t)k1 << 32) | k0;
    uint64_t subseq = ((uint64_t)c3 << 32) | c2;
    uint64_t offset = ((uint64_t)c1 << 32) | c0;
    at::philox_engine eng(seed, subseq, 0);
    eng.set_offset(offset);
    unsigned a = eng(), b = eng(), c = eng(), d = eng();
    printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PhiloxRNGEngine.h not shipped with this torch")
    return inc


@pytest.fixture(scope="module")
def torch_philox():
    inc = _torch_include()
    d = tempfile.mkdtemp(prefix="philox_kat_")
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cannot compile the PyTorch Philox harness: " + r.stderr[-400:])

    def run(ctr, key):
        ctr = np.asarray(ctr, dtype=np.uint32).reshape(-1, 4)
        key = np.asarray(key, dtype=np.uint32).reshape(-1, 2)
        lines = [str(ctr.shape[0])]
        for c, k in zip(ctr, key):
            lines.append(" ".join(str(int(v)) for v in (*c, *k)))
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout
        return np.array([[int(v) for v in ln.split()] for ln in out.strip().splitlines()],
                        dtype=np.uint32)

    return run


def _oracle_rows(ctr, key):
    return np.concatenate([oracle.philox4x32_10(c[None], k) for c, k in zip(ctr, key)])


def test_corner_counters_match_torch_engine(torch_philox):
    m = 0xFFFFFFFF
    ctr = np.array([[0, 0, 0, 0], [m, m, m, m], [1, 0, 0, 0], [0, 0, 0, 1],
                    [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint32)
    key = np.array([[0, 0], [m, m], [0, 0], [1, 0], [0xA4093822, 0x299F31D0]], dtype=np.uint32)
    np.testing.assert_array_equal(_oracle_rows(ctr, key), torch_philox(ctr, key))


def test_random_counters_match_torch_engine(torch_philox):
    rng = np.random.default_rng(20170913)
    ctr = rng.integers(0, 2 ** 32, size=(400, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(400, 2), dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(_oracle_rows(ctr, key), torch_philox(ctr, key))


def test_counter_layout_as_used_by_metropolis_matches_torch_engine(torch_philox):
    # counters of the form (q, t, r, purpose<<28 | colour<<27 | instance), key = seed split
    seed = 0x0123456789ABCDEF
    key = np.array([[seed & 0xFFFFFFFF, seed >> 32]] * 64, dtype=np.uint32)
    q = np.arange(64, dtype=np.uint32)
    ctr = np.stack([q, q * 7 + 3, q % 5, (0 << 28) | (1 << 27) | (q % 3)], axis=1).astype(np.uint32)
    np.testing.assert_array_equal(_oracle_rows(ctr, key), torch_philox(ctr, key))


def test_output_words_are_uniform():
    # 2^16 words: each byte value histogram and the top bit are uniform within 5 sigma
    q = np.arange(1 << 14, dtype=np.uint32)
    ctr = np.stack([q, np.zeros_like(q), np.zeros_like(q), np.zeros_like(q)], axis=1)
    w = oracle.philox4x32_10(ctr, [1, 0]).reshape(-1)
    top = (w >> 31).mean()
    assert abs(top - 0.5) < 5 * 0.5 / np.sqrt(w.size)
    hist = np.bincount((w & 0xFF).astype(np.int64), minlength=256)
    chi2 = float(((hist - w.size / 256) ** 2 / (w.size / 256)).sum())
    assert chi2 < 255 + 6 * np.sqrt(2 * 255)
