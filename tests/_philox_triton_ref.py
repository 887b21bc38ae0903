"""Reference Philox4x32-10 words from Triton's own implementation, run in Triton's
CPU interpreter.  Used by the oracle pins as an implementation of the SC'11
generator that this project did not write.  Run as a subprocess (the interpreter
switch must be set before Triton is imported):

    TRITON_INTERPRET=1 python _philox_triton_ref.py < [[seed, c0, c1, c2, c3], ...]

prints a JSON list of [w0, w1, w2, w3] (uint32) per input line."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(seed, c0, c1, c2, c3, out_ptr):
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 0, a)
    tl.store(out_ptr + 1, b)
    tl.store(out_ptr + 2, c)
    tl.store(out_ptr + 3, d)


def main():
    reqs = json.load(sys.stdin)
    res = []
    for seed, c0, c1, c2, c3 in reqs:
        o32 = torch.zeros(4, dtype=torch.int32)
        # counters are passed as 32-bit values (bit patterns), the seed as 64-bit
        def s32(x):
            return x - (1 << 32) if x >= (1 << 31) else x
        _philox_kernel[(1,)](seed, s32(c0), s32(c1), s32(c2), s32(c3), o32)
        res.append([int(v) & 0xFFFFFFFF for v in o32.tolist()])
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
