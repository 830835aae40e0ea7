"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped
sign, a wrong shift, a dropped clamp, a swapped operand, a wrong constant, a
wrong draw word) and runs tests/test_oracle_pins.py against that copy in a
subprocess.  The mistake must make at least one pin fail.  Nothing here
touches the real oracle or the CUDA library."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file, original text, planted text)
MUTANTS = [
    ("delta sign flipped", "fsb_oracle.c",
     "return f->currentObjective - f->prevObjective;",
     "return f->prevObjective - f->currentObjective;"),
    ("draw mapped with 23 bits", "fsb_oracle.c",
     "real u = (real)(r >> 8) * (real)0x1p-24;",
     "real u = (real)(r >> 9) * (real)0x1p-23;"),
    ("pond clamp dropped", "fsb_oracle.c",
     "f->x = clamp_r(nx, -P, P);", "f->x = nx;"),
    ("dy drawn from the dx word", "fsb_oracle.c",
     "real ny = f->y + centred_uniform(r1) * s;", "real ny = f->y + centred_uniform(r0) * s;"),
    ("weight cap doubled", "fsb_oracle.c",
     "return clamp_r(w + delta / M, wmin, wmax);",
     "return clamp_r(w + delta / M, wmin, (real)2 * wmax);"),
    ("S_x summed over y", "fsb_oracle.c",
     "csum_add_product(&sx, w, x);", "csum_add_product(&sx, w, y);"),
    ("S_w counts fish", "fsb_oracle.c",
     "csum_add(&sw, w);", "csum_add(&sw, 1.0);"),
    ("objective uses x*y", "fsb_oracle.c",
     "return sqrt_r(x * x + y * y);", "return sqrt_r(x * x + x * y);"),
    ("eat() statistic as cur - prev", "fsb_oracle.c",
     "double diff = (double)(school[i].prevObjective -\n"
     "                                   school[i].currentObjective);",
     "double diff = (double)(school[i].currentObjective -\n"
     "                                   school[i].prevObjective);"),
    ("mode-1 initial weight offset", "fsb_oracle.c",
     "f->weight = w0 * ((real)0.5 + u2);", "f->weight = w0 * ((real)0.25 + u2);"),
    ("init y from the x word", "fsb_oracle.c",
     "f->y = centred_uniform(r[1]) * P;", "f->y = centred_uniform(r[0]) * P;"),
    ("eating when M = 0", "fsb_oracle.c",
     "if (cfg->feed_mode == 0 && M > 0.0) {", "if (cfg->feed_mode == 0 && M >= 0.0) {"),
    ("weighted swim ignores w0", "fsb_oracle.c",
     "return (w / w0) * s;", "return w * s;"),
    ("paper feeding normalised by max|delta|", "fsb_oracle.c",
     "const real Er = (real)eat_max;", "const real Er = (real)M;"),
    ("school id added instead of xor", "philox.c",
     "ctr[1] = (uint32_t)(i >> 32) ^ cfg->school_id;",
     "ctr[1] = (uint32_t)(i >> 32) + cfg->school_id;"),
    ("Weyl constant off by one", "philox.c",
     "#define PHILOX_WEYL_0  0x9E3779B9u", "#define PHILOX_WEYL_0  0x9E3779B8u"),
    ("both fish of a pair take words 0 and 1", "philox.c",
     "out[0] = r[2 * half];\n    out[1] = r[2 * half + 1];",
     "out[0] = r[0];\n    out[1] = r[1];"),
    # collective movements (fish-school search variant)
    ("school contracts when its weight fell", "fsb_oracle.c",
     "const int contract = sw > w_before;", "const int contract = sw < w_before;"),
    ("instinctive vector over every fish", "fsb_oracle.c",
     "                if (g > 0) {\n                    nx += grid_term",
     "                if (g == g) {\n                    nx += grid_term"),
    ("grid terms truncated", "fsb_oracle.c",
     "return llrint((double)v * ldexp(1.0, k));",
     "return (long long)((double)v * ldexp(1.0, k));"),
    ("grid exponents swapped in the quotient", "fsb_oracle.c",
     "ix = (real)ldexp((double)nx / (double)den, kg - kp);",
     "ix = (real)ldexp((double)nx / (double)den, kp - kg);"),
    ("objective not updated after the collective moves", "fsb_oracle.c",
     "                school[i].currentObjective = objective(school[i].x, school[i].y);\n"
     "            if (stats) {",
     "                (void)0;\n            if (stats) {"),
    ("both fish of a pair take volitive word 0", "philox.c",
     "return r[i & 1u];", "return r[0];"),
]


@pytest.mark.parametrize("name,src,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, src, old, new, tmp_path):
    parent = tmp_path / "mutant"
    shutil.copytree(os.path.join(ROOT, "oracle"), parent / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = parent / "oracle" / src
    text = path.read_text()
    assert text.count(old) == 1, "the mutation no longer matches the oracle source: %s" % name
    path.write_text(text.replace(old, new))
    env = dict(os.environ, FSB_MUTANT_ORACLE_PARENT=str(parent))
    proc = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
         "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # the copy was the oracle the pins ran on
    assert (parent / "oracle" / "_build" / "libfsb_oracle.so").exists(), proc.stdout[-2000:]
    assert proc.returncode != 0, "no pin caught: %s\n%s" % (name, proc.stdout[-1500:])


def test_unchanged_copy_passes_every_pin(tmp_path):
    """Control: the same harness on an unmodified copy passes, so a failure
    above comes from the planted mistake."""
    parent = tmp_path / "copy"
    shutil.copytree(os.path.join(ROOT, "oracle"), parent / "oracle",
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    env = dict(os.environ, FSB_MUTANT_ORACLE_PARENT=str(parent))
    proc = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
         "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert (parent / "oracle" / "_build" / "libfsb_oracle.so").exists()
    assert proc.returncode == 0, proc.stdout[-2000:]
