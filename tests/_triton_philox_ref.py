"""Philox4x32-10 words from Triton's own implementation, run by Triton's CPU
interpreter.  Used by tests/test_oracle_philox.py as an independent reference
for the oracle's Philox (the Random123 known-answer vectors are not available
offline).  Usage: python _triton_philox_ref.py IN.npy OUT.npy SEED"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402,F401
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_words(c_ptr, o_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.random.philox(seed, c0, c1, c2, c3, 10)
    tl.store(o_ptr + 4 * i, a)
    tl.store(o_ptr + 4 * i + 1, b)
    tl.store(o_ptr + 4 * i + 2, c)
    tl.store(o_ptr + 4 * i + 3, d)


def main():
    ctr = np.load(sys.argv[1]).astype(np.uint32)
    seed = int(sys.argv[3])
    n = ctr.shape[0]
    out = torch.zeros(n * 4, dtype=torch.uint32)
    inp = torch.from_numpy(ctr.view(np.int32).ravel().copy()).view(torch.uint32)
    _philox_words[(1,)](inp, out, seed, N=n)
    np.save(sys.argv[2], out.numpy().reshape(n, 4))


if __name__ == "__main__":
    main()
