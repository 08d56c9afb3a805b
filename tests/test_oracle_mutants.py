"""The oracle's pins catch plausible mistakes in the oracle (CPU only).

Each mutant is oracle.c with one planted mistake of the kind a hand-written
reference might contain: a dropped term, a wrong sign, a wrong index or
shift, a transposed operand or offset, a missing reduction or scale factor.
The mutant is compiled on its own and the pin suites (tests that check the
oracle against closed forms, worked examples, brute force and exact big-
integer products, never against the CUDA path) run against it; every
mutant must make them fail.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PIN_SUITES = ["tests/test_oracle_pins.py", "tests/test_paper_readings.py"]

# (name, text in oracle.c, replacement); every occurrence is replaced.
MUTANTS = [
    ("mulmod_32bit_product", "return (uint32_t)(((uint64_t)a * b) % p);", "return (uint32_t)((a * b) % p);"),
    ("powmod_base_times_a", "base = (base * base) % p;", "base = (base * a) % p;"),
    ("powmod_bit_test_inverted", "if (e & 1) result", "if (!(e & 1)) result"),
    ("invmod_bezout_sign", "tmp = old_s - q * s;", "tmp = old_s + q * s;"),
    ("setup_pprime_sign", "uint64_t rr = OR_R * r_inv - 1;", "uint64_t rr = OR_R * r_inv + 1;"),
    ("setup_r2_not_squared", "out->r2_mod_p = or_mulmod(out->r_mod_p, out->r_mod_p, p);",
     "out->r2_mod_p = out->r_mod_p;"),
    ("to_mont_shift_31", "(((uint64_t)a << 32) % c->p)", "(((uint64_t)a << 31) % c->p)"),
    ("from_mont_times_r", "return or_mulmod(x, c->r_inv, c->p);", "return or_mulmod(x, c->r_mod_p, c->p);"),
    ("mont_mul_rinv_dropped", "return or_mulmod(or_mulmod(x, y, c->p), c->r_inv, c->p);",
     "return or_mulmod(x, y, c->p);"),
    ("mont_fma_subtracts", "((uint64_t)or_mont_mul(c, x, y) + z) % c->p",
     "((uint64_t)or_mont_mul(c, x, y) + c->p - z) % c->p"),
    ("mont_fma_unreduced", "(uint32_t)(((uint64_t)or_mont_mul(c, x, y) + z) % c->p)",
     "(uint32_t)((uint64_t)or_mont_mul(c, x, y) + z)"),
    ("primitive_root_last_factor_dropped", "if (m > 1) factors[nf++] = m;", "(void)0;"),
    ("primitive_root_search_from_3", "for (uint32_t g = 2; g < p; g++)", "for (uint32_t g = 3; g < p; g++)"),
    ("root_of_unity_inverse_ignored", "return inverse ? (uint32_t)or_invmod(w, p) : w;", "return w;"),
    ("root_of_unity_half_order", "uint32_t w = or_powmod(or_primitive_root(p), (p - 1) / n, p);",
     "uint32_t w = or_powmod(or_primitive_root(p), (p - 1) / n * 2, p);"),
    ("dft_index_sum", "wpow[(uint64_t)j * k % n]", "wpow[((uint64_t)j + k) % n]"),
    ("dft_inverse_unscaled", "out[k] = inverse ? or_mulmod((uint32_t)acc, ninv, p) : (uint32_t)acc;",
     "out[k] = (uint32_t)acc;"),
    ("ntt_difference_sign", "out[k + half] = (uint32_t)(((uint64_t)e + p - o) % p);",
     "out[k + half] = (uint32_t)(((uint64_t)e + o) % p);"),
    ("ntt_twiddle_step_w2", "wk = or_mulmod(wk, w, p);", "wk = or_mulmod(wk, w2, p);"),
    ("ntt_odd_half_offset", "ntt_rec(p, x + stride, 2 * stride, half, w2, out + half);",
     "ntt_rec(p, x + 1, 2 * stride, half, w2, out + half);"),
    ("ntt_inverse_unscaled", "for (size_t k = 0; k < n; k++) out[k] = or_mulmod(out[k], ninv, p);",
     "(void)ninv;"),
    ("schoolbook_b_reversed", "or_mulmod(a[i], b[j], p)", "or_mulmod(a[i], b[lb - 1 - j], p)"),
    ("polymul_ntt_size_one_short", "while (n < lc) n <<= 1;", "while (n + 1 < lc) n <<= 1;"),
    ("polymul_ntt_squares_a", "fa[k] = or_mulmod(fa[k], fb[k], p);", "fa[k] = or_mulmod(fa[k], fa[k], p);"),
    ("polymul_batch_b_at_a_offset", "b + b_off[i]", "b + a_off[i]"),
    ("primitive_root_trial_bound", "(uint64_t)q * q <= m", "(uint64_t)q * q < m"),
    ("ninv_of_n_plus_1", "or_invmod(n % p, p)", "or_invmod((n + 1) % p, p)"),
    ("setup_accepts_odd_above_2_31", "p >= 0x80000000u) return -1;", "p == 0xFFFFFFFFu) return -1;"),
    ("invmod_negative_kept", "if (old_s < 0) old_s += (int64_t)m;", "(void)0;"),
    ("schoolbook_no_accumulate", "c[i + j] = (uint32_t)(((uint64_t)c[i + j] + or_mulmod(a[i], b[j], p)) % p);",
     "c[i + j] = or_mulmod(a[i], b[j], p);"),
    ("mulmod_vec_squares_x", "out[i] = or_mulmod(x[i], y[i], p);", "out[i] = or_mulmod(x[i], x[i], p);"),
    ("tft_needed_entries_rounded_down", "const size_t need = (l + h - 1) / h * h;",
     "const size_t need = l / h * h + (l < h ? h : 0);"),
    ("tft_twiddle_not_bit_reversed", "or_powmod(w, brev_bits(b / (2 * h), s) * h, p)", "or_powmod(w, (b / (2 * h)) * h, p)"),
    ("itft_right_tail_plus", "a[h + j] = submod(a[j], or_mulmod(2 % p, or_mulmod(r, a[h + j], p), p), p);",
     "a[h + j] = addmod(a[j], or_mulmod(2 % p, or_mulmod(r, a[h + j], p), p), p);"),
    ("itft_half_dropped", "a[j] = or_mulmod(addmod(u, v, p), inv2, p);", "a[j] = addmod(u, v, p);"),
    ("itft_left_tail_minus", "for (size_t j = l; j < h; j++) a[j] = addmod(a[j], or_mulmod(r, a[h + j], p), p);",
     "for (size_t j = l; j < h; j++) a[j] = submod(a[j], or_mulmod(r, a[h + j], p), p);"),
    ("itft_twiddle_of_parent_level", "((uint64_t)1 << (log2n - s - 1))", "((uint64_t)1 << (log2n - s))"),
    ("polymul_tft_b_transform_into_a", "if (rc == 0) rc = or_tft(p, t, l, k, pb);",
     "if (rc == 0) rc = or_tft(p, t, l, k, pa);"),
]


def _source():
    with open(os.path.join(ORACLE_DIR, "oracle.c")) as f:
        return f.read()


def _run_mutant(name, old, new, workdir):
    src = _source()
    assert old in src, "mutant %s: text not found in oracle.c" % name
    path_c = os.path.join(workdir, name + ".c")
    path_so = os.path.join(workdir, name + ".so")
    with open(path_c, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-w", "-I", ORACLE_DIR,
                    "-o", path_so, path_c], check=True)
    env = dict(os.environ, ORACLE_LIB=path_so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                       + PIN_SUITES, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode, (r.stdout + r.stderr)[-400:]


def test_mutant_list_applies():
    src = _source()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new in MUTANTS:
        assert old in src, name
        assert old != new, name


def test_pins_kill_every_mutant(tmp_path):
    """Every planted mistake makes the pin suites fail (a failed test, or a
    crash of the test process on a mutant that reads out of bounds); the
    unmutated build passing the same harness shows the failures come from
    the mistakes."""
    workers = max(1, min(len(MUTANTS), os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda m: _run_mutant(m[0], m[1], m[2], str(tmp_path)), MUTANTS))
    survivors = [(name, tail) for name, rc, tail in results if rc == 0]
    assert not survivors, survivors


def test_unmutated_oracle_passes_the_same_way(tmp_path):
    """The harness itself: the unchanged source, built the same way, passes."""
    name, rc, tail = _run_mutant("identity", "#include \"oracle.h\"", "#include \"oracle.h\"", str(tmp_path))
    assert rc == 0, tail
