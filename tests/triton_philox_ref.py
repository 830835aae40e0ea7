"""Philox4x32-10 words from Triton's library implementation, run on the CPU
through Triton's interpreter.  Used only as an independent reference for the
oracle's generator (tests/test_oracle_pins.py runs it in a subprocess so the
interpreter switch cannot leak into other tests).

stdin:  JSON list of [c0, c1, c2, c3, seed64]
stdout: JSON list of [r0, r1, r2, r3]
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(out, c0p, c1p, c2p, c3p, seed, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c0p + offs, mask=m)
    c1 = tl.load(c1p + offs, mask=m)
    c2 = tl.load(c2p + offs, mask=m)
    c3 = tl.load(c3p + offs, mask=m)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out + offs * 4 + 0, r0, mask=m)
    tl.store(out + offs * 4 + 1, r1, mask=m)
    tl.store(out + offs * 4 + 2, r2, mask=m)
    tl.store(out + offs * 4 + 3, r3, mask=m)


def main():
    rows = json.load(sys.stdin)
    by_seed = {}
    for idx, (c0, c1, c2, c3, seed) in enumerate(rows):
        by_seed.setdefault(seed, []).append((idx, c0, c1, c2, c3))
    result = [None] * len(rows)
    for seed, items in by_seed.items():
        n = len(items)
        block = 1 << max(0, (n - 1).bit_length())
        cols = [torch.tensor([it[k] for it in items] + [0] * (block - n),
                             dtype=torch.uint32) for k in range(1, 5)]
        out = torch.zeros(4 * block, dtype=torch.uint32)
        _philox_kernel[(1,)](out, cols[0], cols[1], cols[2], cols[3],
                             seed, n, BLOCK=block)
        words = out.tolist()
        for j, it in enumerate(items):
            result[it[0]] = [int(w) & 0xFFFFFFFF for w in words[4 * j:4 * j + 4]]
    json.dump(result, sys.stdout)


if __name__ == "__main__":
    main()
