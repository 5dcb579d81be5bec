"""Plant plausible mistakes in copies of the oracle and check the pins catch them.

Each mutant is a textual edit of ``oracle/oracle.c`` (a flipped sign, a dropped
twiddle, a transposed index, a wrong root power, ...), compiled with gcc into a
temporary library and run against a compact battery of the pins from
``test_oracle_pins.py`` in a child process (a mutant that crashes counts as
caught).  The unmodified source must pass the same battery.
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "root_sign_flipped": ("r[m].im = (double)sign * sin(a);", "r[m].im = -(double)sign * sin(a);"),
    "ct_twiddle_dropped": ("tmp[l2] = cmul(y[l2 * m + k1], rootN[((l2 * k1) % n) * scale]);",
                           "tmp[l2] = y[l2 * m + k1];"),
    "ct_output_index_transposed": ("y[k1 + k2 * m] = acc;", "y[k1 * p + k2] = acc;"),
    "ct_subsequence_order_reversed": ("dft_ct_rec(m, N, rootN, x + l2 * xs, p * xs, y + l2 * m, tmp);",
                                      "dft_ct_rec(m, N, rootN, x + (p - 1 - l2) * xs, p * xs, y + l2 * m, tmp);"),
    "ct_radix_root_wrong_power": ("rootN[(((l2 * k2) % p) * m) * scale]", "rootN[(((l2 * k2) % p)) * scale]"),
    "ct_prime_leaf_scale_dropped": ("cmul(x[l * xs], rootN[((l * k) % n) * scale]);",
                                    "cmul(x[l * xs], rootN[((l * k) % n)]);"),
    "direct_index_shifted": ("roots[(l * k) % n]", "roots[(l * k + l) % n]"),
    "multidim_last_dim_skipped": ("        for (int d = 0; d < jb->rank; ++d) {\n            int64_t nd",
                                  "        for (int d = 0; d < jb->rank - 1; ++d) {\n            int64_t nd"),
    "gather_uses_row_major_temp_wrong": ("off += (r % jb->n[d]) * jb->is[d];",
                                        "off += (r % jb->n[d]) * jb->is[jb->rank - 1 - d];"),
    "vector_offset_dims_swapped": ("a += i * jb->vis[d];", "a += i * jb->vis[jb->vrank - 1 - d];"),
}

BATTERY = textwrap.dedent(r'''
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle, fft_inputs
    lib = oracle.open_library(LIB)

    def rel(a, b):
        return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)

    def one(n, x, sign=-1, algo="auto"):
        return oracle.dft(x, [(n, 1, 1)], [], sign, algo=algo, threads=2, lib=lib)

    bad = []
    # closed form: delta at l0 -> w_n^{l0 k}, on both algorithms
    for n in (8, 12, 30, 5000, 10007):
        for algo in ("direct", "ct"):
            if algo == "direct" and n > 4096:
                continue
            x = np.zeros(n, complex); x[1] = 1
            k = np.arange(n)
            if np.max(np.abs(one(n, x, -1, algo) - np.exp(-2j*np.pi*k/n))) > 1e-11:
                bad.append(("delta", n, algo))
    # direct vs Cooley-Tukey, small n
    for n in range(2, 65):
        x = fft_inputs.uniform_c64(n, n).astype(complex)
        if rel(one(n, x, -1, "ct"), one(n, x, -1, "direct")) > 1e-13:
            bad.append(("ct_vs_direct", n)); break
    # independent library routine
    for n in (15, 1000, 7168, 10007, 4 * 10007):
        x = fft_inputs.uniform_c64(n, 3).astype(complex)
        if rel(one(n, x), np.fft.fft(x)) > 1e-12:
            bad.append(("numpy", n))
    # multi-dimensional and strided layouts
    x = fft_inputs.uniform_c64(6 * 10 * 7, 8)
    y = oracle.dft(x, [(6, 70, 70), (10, 7, 7), (7, 1, 1)], [], -1, lib=lib)
    if rel(y, np.fft.fftn(x.astype(complex).reshape(6, 10, 7)).reshape(-1)) > 1e-13:
        bad.append(("fftn",))
    n, b = 16, 5
    x = fft_inputs.uniform_c64(n * b, 24)
    y = oracle.dft(x, [(n, 1, b)], [(b, n, 1)], -1, lib=lib)
    if rel(y.reshape(n, b).T, np.fft.fft(x.astype(complex).reshape(b, n), axis=1)) > 1e-13:
        bad.append(("strided",))
    x = fft_inputs.uniform_c64(4 * 3 * 8, 9)
    y = oracle.dft(x, [(8, 1, 1)], [(4, 24, 24), (3, 8, 8)], -1, lib=lib)
    if rel(y.reshape(12, 8), np.fft.fft(x.astype(complex).reshape(12, 8), axis=1)) > 1e-13:
        bad.append(("vector2",))
    print(bad)
    sys.exit(1 if bad else 0)
''')


def _build(src_text, path):
    c = path + ".c"
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-D_DEFAULT_SOURCE", "-shared", "-fPIC", c,
                           "-o", path, "-lpthread", "-lm"])


def _run_battery(lib_path):
    code = f"ROOT = {ROOT!r}\nLIB = {lib_path!r}\n" + BATTERY
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    return p.returncode, p.stdout + p.stderr


def test_unmodified_oracle_passes_battery(tmp_path):
    lib = str(tmp_path / "lib_orig.so")
    _build(open(SRC).read(), lib)
    rc, out = _run_battery(lib)
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    lib = str(tmp_path / f"lib_{name}.so")
    _build(src.replace(old, new), lib)
    rc, out = _run_battery(lib)
    assert rc != 0, f"mutant {name} survived the pin battery: {out}"
