"""The C-ABI library builds, loads, and exports every entry point include/pmcmc.h declares.
No compute call is made here (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "pmcmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmcmc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ["pmcmc_create", "pmcmc_destroy", "pmcmc_last_error", "pmcmc_gen_noise",
              "pmcmc_solve", "pmcmc_seq_solve", "pmcmc_linearize", "pmcmc_scan",
              "pmcmc_adjoint", "pmcmc_solve_batched", "pmcmc_options_default"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2508_18413_gb300 import build, _lib
    path = build.build()
    lib = C.CDLL(path)
    for n in declared_entry_points():
        assert hasattr(lib, n), f"{n} missing from {path}"
    _lib.load(path)


def test_options_default_without_gpu():
    from paper_2508_18413_gb300 import _lib
    lib = _lib.load()
    o = _lib.pmcmc_options()
    lib.pmcmc_options_default(C.byref(o))
    assert o.jac == 1 and o.precision == 1 and o.gate_grad == 1 and abs(o.atol - 1e-5) < 1e-20


def test_struct_layouts_match_header():
    """The Python mirrors of the C structs have the C sizes (checked against a compiled probe)."""
    from paper_2508_18413_gb300 import _lib
    import subprocess, tempfile
    prog = r'''
#include <stdio.h>
#include "pmcmc.h"
int main(void){printf("%zu %zu %zu %zu\n", sizeof(pmcmc_target), sizeof(pmcmc_options),
 sizeof(pmcmc_result), sizeof(pmcmc_chain_desc)); return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        cfile = os.path.join(d, "p.c")
        open(cfile, "w").write(prog)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), cfile, "-o", exe])
        sizes = list(map(int, subprocess.check_output([exe]).split()))
    assert sizes == [C.sizeof(_lib.pmcmc_target), C.sizeof(_lib.pmcmc_options),
                     C.sizeof(_lib.pmcmc_result), C.sizeof(_lib.pmcmc_chain_desc)]


def test_struct_field_offsets_match_header():
    """Every field of the Python mirrors sits at the C offset (offsetof in a compiled probe), so
    a field added on one side only cannot shift the others unnoticed."""
    from paper_2508_18413_gb300 import _lib
    import subprocess, tempfile
    structs = [("pmcmc_target", _lib.pmcmc_target), ("pmcmc_options", _lib.pmcmc_options),
               ("pmcmc_result", _lib.pmcmc_result), ("pmcmc_chain_desc", _lib.pmcmc_chain_desc)]
    lines = []
    for cname, py in structs:
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    prog = ("#include <stdio.h>\n#include <stddef.h>\n#include \"pmcmc.h\"\nint main(void){\n" +
            "\n".join(lines) + "\nreturn 0;}\n")
    with tempfile.TemporaryDirectory() as d:
        cfile = os.path.join(d, "p.c")
        open(cfile, "w").write(prog)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), cfile, "-o", exe])
        got = dict(l.split() for l in subprocess.check_output([exe]).decode().splitlines())
    for cname, py in structs:
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_options_default_leaves_extensions_off():
    from paper_2508_18413_gb300 import _lib
    lib = _lib.load()
    o = _lib.pmcmc_options()
    lib.pmcmc_options_default(C.byref(o))
    assert o.window == 0 and o.seq_after == 0 and o.engine == 0 and o.sampler == 0


def test_missing_library_fails_loudly(tmp_path):
    """The binding has no CPU path: without the built library it raises instead of computing."""
    import subprocess
    import sys
    code = ("import paper_2508_18413_gb300._lib as L\n"
            "L._lib = None\n"
            f"L.load({str(tmp_path / 'absent.so')!r})\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode != 0 and "no fallback" in r.stderr.replace("\n", " ")


def test_reference_arm_json_contract():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one JSON line with
    the contract's keys and runs without a GPU."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
