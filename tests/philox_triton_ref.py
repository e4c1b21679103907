"""Philox4x32-10 evaluated by Triton's own implementation of the generator
(``triton.language.random.philox_impl``), run by Triton's interpreter on the
CPU. An independent implementation of the published definition (Salmon et
al., SC'11) for the oracle's noise pin: unlike the cuRAND host generator, it
takes all four counter words, so it reaches word 3 (the chain id of the
method's noise counter). Test infrastructure only; the library never uses
Triton.

Run as a script (the interpreter must be switched on before Triton is
imported): reads a uint32 [n][4] counter array and the 64-bit key from
stdin (.npy, then 8 little-endian bytes), writes the uint32 [n][4] output
blocks to stdout (.npy).
"""
import io
import os
import sys

import numpy as np

BLOCK = 128


def main() -> None:
    os.environ["TRITON_INTERPRET"] = "1"
    import torch
    import triton
    import triton.language as tl

    @triton.jit
    def philox_blocks(c_ptr, o_ptr, k_lo, k_hi, n, BLOCK: tl.constexpr):
        offs = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
        msk = offs < n
        c0 = tl.load(c_ptr + 4 * offs + 0, mask=msk).to(tl.uint32, bitcast=True)
        c1 = tl.load(c_ptr + 4 * offs + 1, mask=msk).to(tl.uint32, bitcast=True)
        c2 = tl.load(c_ptr + 4 * offs + 2, mask=msk).to(tl.uint32, bitcast=True)
        c3 = tl.load(c_ptr + 4 * offs + 3, mask=msk).to(tl.uint32, bitcast=True)
        k0 = tl.full((BLOCK,), 0, tl.uint32) + k_lo.to(tl.uint32, bitcast=True)
        k1 = tl.full((BLOCK,), 0, tl.uint32) + k_hi.to(tl.uint32, bitcast=True)
        x0, x1, x2, x3 = tl.random.philox_impl(c0, c1, c2, c3, k0, k1, 10)
        tl.store(o_ptr + 4 * offs + 0, x0.to(tl.int32, bitcast=True), mask=msk)
        tl.store(o_ptr + 4 * offs + 1, x1.to(tl.int32, bitcast=True), mask=msk)
        tl.store(o_ptr + 4 * offs + 2, x2.to(tl.int32, bitcast=True), mask=msk)
        tl.store(o_ptr + 4 * offs + 3, x3.to(tl.int32, bitcast=True), mask=msk)

    data = sys.stdin.buffer.read()
    ctr = np.load(io.BytesIO(data[:-8]))
    key = int.from_bytes(data[-8:], "little")
    n = len(ctr)
    c = torch.from_numpy(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32))
    out = torch.zeros_like(c)
    as_i32 = lambda w: int(np.uint32(w).view(np.int32))
    philox_blocks[(-(-n // BLOCK),)](c, out, as_i32(key & 0xFFFFFFFF), as_i32(key >> 32), n,
                                     BLOCK=BLOCK)
    buf = io.BytesIO()
    np.save(buf, out.numpy().view(np.uint32))
    sys.stdout.buffer.write(buf.getvalue())


if __name__ == "__main__":
    main()
