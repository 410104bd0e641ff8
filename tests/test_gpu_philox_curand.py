"""Second independent pin of the oracle's Philox4x32-10 (Sec. 4): cuRAND's
device-side Philox4_32_10 generator, run on the GPU through a small harness
compiled here with nvcc, must give the oracle's words for the same counter
and key. cuRAND's state takes key = seed and counter = (offset / 4 as a
64-bit number, subsequence as a 64-bit number), so any (counter, key) pair
with a counter below 2^62 in its low half is reachable.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

HARNESS = r"""
#include <curand_kernel.h>
#include <cstdio>
#include <cstdint>
#include <vector>

__global__ void draw(const unsigned long long* seed, const unsigned long long* subseq,
                     const unsigned long long* offset, uint4* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed[i], subseq[i], offset[i], &st);
  out[i] = curand4(&st);
}

int main() {
  int n;
  if (scanf("%d", &n) != 1 || n <= 0 || n > 100000) return 1;
  std::vector<unsigned long long> seed(n), subseq(n), offset(n);
  for (int i = 0; i < n; ++i) {
    unsigned c0, c1, c2, c3, k0, k1;
    if (scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) != 6) return 2;
    seed[i] = ((unsigned long long)k1 << 32) | k0;
    subseq[i] = ((unsigned long long)c3 << 32) | c2;
    offset[i] = 4ull * (((unsigned long long)c1 << 32) | c0);
  }
  unsigned long long *ds, *dq, *dof;
  uint4* dout;
  size_t b = n * sizeof(unsigned long long);
  if (cudaMalloc(&ds, b) || cudaMalloc(&dq, b) || cudaMalloc(&dof, b) || cudaMalloc(&dout, n * sizeof(uint4)))
    return 3;
  cudaMemcpy(ds, seed.data(), b, cudaMemcpyHostToDevice);
  cudaMemcpy(dq, subseq.data(), b, cudaMemcpyHostToDevice);
  cudaMemcpy(dof, offset.data(), b, cudaMemcpyHostToDevice);
  draw<<<(n + 127) / 128, 128>>>(ds, dq, dof, dout, n);
  std::vector<uint4> out(n);
  if (cudaMemcpy(out.data(), dout, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
  for (int i = 0; i < n; ++i) printf("%u %u %u %u\n", out[i].x, out[i].y, out[i].z, out[i].w);
  cudaFree(ds); cudaFree(dq); cudaFree(dof); cudaFree(dout);
  return 0;
}
"""


@pytest.fixture(scope="module")
def curand_philox():
    require_gpu()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "h.cu"), os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a", src, "-o", exe], check=True,
                   capture_output=True)

    def run(ctr, key):
        ctr = np.asarray(ctr, dtype=np.uint32).reshape(-1, 4)
        key = np.asarray(key, dtype=np.uint32).reshape(-1, 2)
        lines = ["%d" % len(ctr)] + ["%d %d %d %d %d %d" % (*c, *k) for c, k in zip(ctr, key)]
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return np.array([[int(v) for v in ln.split()] for ln in r.stdout.strip().splitlines()], dtype=np.uint32)

    yield run
    shutil.rmtree(d, ignore_errors=True)


def test_oracle_philox_matches_curand(curand_philox):
    rng = np.random.default_rng(17)
    n = 2000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] >>= 2  # offset = 4 * (c1:c0) must stay below 2^64
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0xFFFFFFFF, 0x3FFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]]
    key[:4] = [[0, 0], [0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [1, 2]]
    got = curand_philox(ctr, key)
    want = np.stack([oracle.philox4x32_10(c, k)[0] for c, k in zip(ctr, key)])
    np.testing.assert_array_equal(got, want)
