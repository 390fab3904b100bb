"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, compiles circuits on the host, and validates arguments."""
import ctypes
import os
import random
import re

import pytest

import paper_2607_28600_b300 as S
from oracle import symft as osymft
from oracle.circuit import parse as oparse
from paper_2607_28600_b300.workloads import random_near_clifford, rotated_surface_code_memory
from tests.circuits_for_tests import random_clifford_text

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    declared = set()
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            hdr = open(os.path.join(ROOT, "include", name)).read()
            declared |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(symft_\w+)\s*\(", hdr, re.M))
    assert declared == set(S.EXPORTS)
    L = S.lib()
    for name in declared:
        assert hasattr(L, name), name


def test_plan_info_matches_oracle_planner():
    """Without the commutation-aware simplification (which the oracle's plain
    SymFT never applies) the C++ compile step and the oracle plan the same
    instruction stream."""
    for trial in range(25):
        rng = random.Random(900 + trial)
        n = rng.randint(2, 7)
        txt = random_clifford_text(rng, n, 60, rot=0.25)
        p = S.symft_compile(txt, simplify=False)
        o = osymft.Plan(oparse(txt))
        info = p.info
        assert info["k_max"] == o.stats["k_max"]
        for name, cnt in info["n_instr"].items():
            assert cnt == o.stats["hist"].get(name, 0), (trial, name)


@pytest.mark.parametrize("d", [3, 5, 7])
def test_surface_code_plan_counts(d):
    p = S.symft_compile(rotated_surface_code_memory(d, d, 1e-3))
    info = p.info
    c = oparse(rotated_surface_code_memory(d, d, 1e-3))
    assert info["n_qubits"] == c.num_qubits
    assert info["n_records"] == c.num_records and info["n_dets"] == c.num_dets
    assert info["n_channels"] == c.num_channels and info["k_max"] == 0
    # first-round X checks and half of the final data measurements are random
    assert info["n_instr"]["RandomMeas"] == d * d - 1


@pytest.mark.parametrize("d,rounds", [(3, 24), (3, 40), (11, 11), (13, 13)])
def test_long_and_large_record_chains_compile(d, rounds):
    """The compile step turns the record chains into paths (each record at
    most one parent and one child, at most 16 records per path) and the device
    image checks both properties; memories whose stabilizer chains are longer
    than a path (24 and 40 rounds) or large (d = 11, 13) compile with every
    record of the circuit in the plan."""
    p = S.symft_compile(rotated_surface_code_memory(d, rounds, 1e-3))
    info = p.info
    assert info["n_records"] == (d * d - 1) * rounds + d * d
    assert info["sign_xor_terms"] > 0


@pytest.mark.parametrize("text,code", [
    ("H 0\nFOO 1\n", -2),
    ("H 0\nCX 0\n", -1),
    ("M 0\nDETECTOR rec[-2]\n", -1),
    ("X_ERROR(1.5) 0\n", -1),
    ("REPEAT 2 {\nH 0\n", -1),
    ("R_PAULI(0.1) X0*Z0\n", -1),
    ("MPP X0*Q1\n", -1),
])
def test_compile_errors(text, code):
    with pytest.raises(S.SymftError) as ei:
        S.symft_compile(text)
    assert ei.value.code == code


def test_sample_argument_errors_before_any_device_work():
    p = S.symft_compile("H 0\nM 0\n")
    with pytest.raises(S.SymftError) as ei:
        S.symft_sample_ex(p, 0, 1)
    assert ei.value.code == -3
    with pytest.raises(S.SymftError) as ei:
        S.symft_sample_ex(p, 10, 1, shot_offset=64)
    assert ei.value.code == -3
    with pytest.raises(S.SymftError) as ei:
        S.symft_sample_ex(p, 10, 1, shot_offset=256)    # not a whole 512-shot noise block
    assert ei.value.code == -3 and "512" in str(ei.value)
    with pytest.raises(S.SymftError) as ei:
        S.symft_sample_ex(p, 10, 1, precision=7)
    assert ei.value.code == -3


def test_null_arguments():
    L = S.lib()
    assert L.symft_compile(None, None) == -3
    assert L.symft_plan_info(None, None) == -3
    L.symft_plan_free(None)
    assert L.symft_sample(None, 1, 1, None, None, None, None) == -3


def test_capacity_error_for_wide_active_state():
    # 26 independent T rotations on |+> promote 26 coordinates
    txt = "H " + " ".join(map(str, range(26))) + "\n" + "T " + " ".join(map(str, range(26))) + "\nM 0\n"
    with pytest.raises(S.SymftError) as ei:
        S.symft_compile(txt)
    assert ei.value.code == -4


def test_repeat_and_generators_compile():
    txt = "R 0 1\nREPEAT 3 {\nH 0\nCX 0 1\nMR 1\nDETECTOR rec[-1]\n}\nM 0\n"
    p = S.symft_compile(txt)
    assert p.info["n_records"] == 4 and p.info["n_dets"] == 3
    p2 = S.symft_compile(random_near_clifford(20, 30, 6, seed=3))
    assert p2.info["n_qubits"] == 20


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the C sizes and field offsets."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"symft_options": S._Options, "symft_info": S._Info,
               "symft_sample_args": S._SampleArgs, "symft_job": S._Job, "symft_peaks": S._Peaks}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "symft.h"', '#include "symft_peaks.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('  printf("SHOT_ALIGN %d\\n", SYMFT_SHOT_ALIGN);')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                   text=True).stdout.splitlines())
    assert int(got["SHOT_ALIGN"]) == S.SHOT_ALIGN
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_listed_postselection_validation():
    txt = "M 0\nDETECTOR rec[-1]\nM 1\nDETECTOR rec[-1]\n"
    S.symft_compile(txt, postselect=S.POSTSELECT_LISTED, post_dets=[1, 1, 0])
    S.symft_compile(txt, postselect=S.POSTSELECT_LISTED, post_dets=[])
    with pytest.raises(S.SymftError) as ei:
        S.symft_compile(txt, postselect=S.POSTSELECT_LISTED, post_dets=[2])
    assert ei.value.code == -3 and "out of range" in str(ei.value)
    with pytest.raises(S.SymftError) as ei:
        S.symft_compile(txt, postselect=3)
    assert ei.value.code == -3
    opt = S._Options()
    opt.postselect = S.POSTSELECT_LISTED
    opt.n_post_dets = 2            # no list given
    h = ctypes.c_void_p()
    assert S.lib().symft_compile_ex(txt.encode(), ctypes.byref(opt), ctypes.byref(h)) == -3


def test_active_measurement_ordinals_match_the_oracle_plan():
    for trial in range(10):
        rng = random.Random(700 + trial)
        txt = random_clifford_text(rng, rng.randint(2, 7), 60, rot=0.3)
        p = S.symft_compile(txt, simplify=False)
        o = osymft.Plan(oparse(txt))
        want = [ins["t"] for ins in o.instrs if ins["op"] in ("ActiveDiagMeas", "ActivePairMeas")]
        assert p.active_meas() == want
        assert len(want) == p.info["n_causal"]
    assert S.symft_compile("H 0\nM 0\n").active_meas() == []
