"""Plants plausible mistakes in a copy of the oracle's C source and checks that the
library-routine pin (every window equals numpy.fft.fft2 of its patch, Section 4.1 Eq. 2)
rejects every mutant.  Runs on the CPU only; the committed oracle is never modified."""
import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle", "swdft2d_oracle.c")

# (name, method, original text, mutated text)
MUTANTS = [
    ("exponent_sign", 0, "w[2 * j + 1] = -sin(ang);", "w[2 * j + 1] = sin(ang);"),
    ("dropped_imag_term", 0,
     "(q1 + j1));\n                    sr += v[0] * er - v[1] * ei;",
     "(q1 + j1));\n                    sr += v[0] * er;"),
    ("kernel_product_sign", 0, "double er = e0[0] * e1[0] - e0[1] * e1[1];\n                    double ei = e0[0] * e1[1] + e0[1] * e1[0];",
     "double er = e0[0] * e1[0] + e0[1] * e1[1];\n                    double ei = e0[0] * e1[1] + e0[1] * e1[0];"),
    ("transposed_operand", 0, "const double *v = x + 2 * ((q0 + j0) * N1 + (q1 + j1));",
     "const double *v = x + 2 * ((q0 + j1 % n0) * N1 + (q1 + j0 % n1));"),
    ("missing_scale", 0, "out[2 * (k0 * n1 + k1)] = c * sr;\n            out[2 * (k0 * n1 + k1) + 1] = c * si;\n        }\n    }\n}\n\n/* One window by the row-column",
     "out[2 * (k0 * n1 + k1)] = sr;\n            out[2 * (k0 * n1 + k1) + 1] = si;\n        }\n    }\n}\n\n/* One window by the row-column"),
    ("separable_dropped_row_offset", 1, "const double *row = x + 2 * ((q0 + j0) * N1 + q1);",
     "const double *row = x + 2 * (q0 * N1 + q1);"),
    ("separable_swapped_lengths", 1, "const double *e = w0 + 2 * (((int64_t)j0 * k0) % n0);\n                const double *v = z + 2 * (j0 * n1 + k1);",
     "const double *e = w0 + 2 * (((int64_t)j0 * k1) % n0);\n                const double *v = z + 2 * (j0 * n1 + k1);"),
]


def _fft2_windows(x, n0, n1):
    P0, P1 = x.shape[0] - n0 + 1, x.shape[1] - n1 + 1
    return np.stack([[np.fft.fft2(x[i:i + n0, j:j + n1]) for j in range(P1)]
                     for i in range(P0)]) / math.sqrt(n0 * n1)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name,method,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(tmp_path, name, method, orig, mut):
    src = open(ORACLE_SRC).read()
    assert src.count(orig) == 1, f"mutation site for {name} not found exactly once"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(orig, mut))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(mpath), "-lm"],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    lib.swo_swdft2d.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_void_p]
    rng = np.random.default_rng(7)
    N0, N1, n0, n1 = 9, 13, 4, 8
    x = np.ascontiguousarray(rng.standard_normal((N0, N1)) + 1j * rng.standard_normal((N0, N1)))
    out = np.empty((N0 - n0 + 1, N1 - n1 + 1, n0, n1), dtype=np.complex128)
    rc = lib.swo_swdft2d(x.ctypes.data, N0, N1, n0, n1, 1 / math.sqrt(n0 * n1), method, 1,
                         out.ctypes.data)
    assert rc == 0
    err = np.abs(out - _fft2_windows(x, n0, n1)).max()
    assert err > 1e-6, f"mutant {name} was not caught (err {err})"
