"""The tensor-core row GEMM's A operand (csrc/tc_kernels.cu, tc_row_kernel), replayed on the CPU.

A[m][k] = x[q1_0 + m + k] (Re x then Im x for complex input) is a Hankel matrix.  The kernel
stores eight copies of the staged input row shifted by s = 0..7 elements (unit u of copy s =
x[8u + s .. 8u + s + 7] at byte (8u + s) 16; complex input interleaves Re and Im unit rows)
and reads it as an MN-major operand: for the 16-wide k-step ks the descriptor starts at one
unit row and steps one unit row (or two) along M and along K.  These tests write the copies
exactly as the kernel's builder loop does, read every (m, k) back through the descriptor's
address rule (MN-major, no swizzle: start + (m / 8) SBO + (k / 8) LBO + (k mod 8) 16 +
(m mod 8) 2), and check each element is the x value the product needs and every address lies
inside the copies.  Rows of A with k past the window meet zero rows of B, so any finite value
is correct there.
"""
import pytest

TC_CH = 128


def tcr_K(m1, cplx):
    k = (2 if cplx else 1) << m1
    return max(16, k)


def units(m1, cplx):
    kp = (1 << m1) if cplx else tcr_K(m1, False)
    return TC_CH // 8 + (kp + 7) // 8


def copy_bytes(m1, cplx):
    return (2 if cplx else 1) * units(m1, cplx) * 128


def build(m1, cplx):
    """Shared memory of one set of copies: byte -> (part, staged column) or 'zero'."""
    n1 = 1 << m1
    W = TC_CH + n1
    U = units(m1, cplx)
    mem = {}
    parts = 2 if cplx else 1
    for e in range(parts * U * 8):
        part = e // (U * 8) if cplx else 0
        us = e - part * U * 8
        u, sh = us >> 3, us & 7
        off = ((2 * u + part) if cplx else u) * 128 + sh * 16
        for j in range(8):
            c = 8 * u + sh + j
            val = (part, c) if c < W else "zero"
            for b in range(2):
                assert off + 2 * j + b not in mem, "two slots written to one byte"
                mem[off + 2 * j + b] = val
    assert max(mem) < copy_bytes(m1, cplx)
    return mem


def descriptor(m1, cplx, ks):
    """(start byte, LBO, SBO) of k-step ks, as the kernel computes them."""
    n1 = 1 << m1
    sbo = 256 if cplx else 128
    lbo = 128 if (cplx and n1 == 8) else sbo
    k0 = 16 * ks
    row = (0 if n1 == 8 else 2 * ((k0 % n1) // 8) + k0 // n1) if cplx else k0 // 8
    return row * 128, lbo, sbo


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m1", [3, 4, 5, 6])
def test_hankel_operand_reads_the_right_x(m1, cplx):
    n1 = 1 << m1
    K = tcr_K(m1, cplx)
    mem = build(m1, cplx)
    for ks in range(K // 16):
        start, lbo, sbo = descriptor(m1, cplx, ks)
        for m in range(TC_CH):
            for kl in range(16):
                k = 16 * ks + kl
                addr = start + (m // 8) * sbo + (kl // 8) * lbo + (kl % 8) * 16 + (m % 8) * 2
                assert 0 <= addr and addr + 1 < copy_bytes(m1, cplx)
                got = mem[addr]
                assert mem[addr + 1] == got
                if cplx:
                    want = (0, m + k) if k < n1 else ((1, m + k - n1) if k < 2 * n1 else None)
                else:
                    want = (0, m + k) if k < n1 else None
                if want is None:
                    continue            # meets a zero row of B
                assert got == want, (m, k, got, want)


def test_planted_stride_mistake_is_caught():
    """The complex n1 = 8 step with the M stride as its K stride reads Re where Im belongs."""
    m1, cplx = 3, True
    mem = build(m1, cplx)
    start, lbo, sbo = descriptor(m1, cplx, 0)
    bad = 0
    for m in range(TC_CH):
        for kl in range(8, 16):
            addr = start + (m // 8) * sbo + (kl // 8) * sbo + (kl % 8) * 16 + (m % 8) * 2
            if addr + 1 >= copy_bytes(m1, cplx) or mem.get(addr) != (1, m + kl - 8):
                bad += 1
    assert bad > 0
