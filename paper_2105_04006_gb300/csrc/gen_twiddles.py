"""Writes lsp_twiddles.inc: e^{2 pi i j / 256}, j = 0..255, as {cos, sin}
pairs of doubles, each correctly rounded from a 60-digit evaluation
(mpmath).  The table feeds sincos_fixed64 in lsp_common.cuh; run this file to
regenerate it (the build uses the committed copy)."""
import os

import mpmath

mpmath.mp.dps = 60
HERE = os.path.dirname(os.path.abspath(__file__))
lines = ["// e^{2 pi i j / 256}, j = 0..255, {cos, sin}: written by gen_twiddles.py (do not edit)"]
for j in range(256):
    x = mpmath.mpf(2 * j) / 256  # the angle in units of pi (exact zeros and ones where due)
    c, s = float(mpmath.cospi(x)), float(mpmath.sinpi(x))
    lines.append(f"{{{c!r}, {s!r}}},")
with open(os.path.join(HERE, "lsp_twiddles.inc"), "w") as f:
    f.write("\n".join(lines) + "\n")
