"""The C-ABI library loads, exports every entry point its header declares,
and its host-only planner agrees with the oracle's sizing (no GPU needed)."""
import os
import re

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "bolt.h")).read()
    return sorted(set(re.findall(r"BOLT_API\s+(?:const\s+)?\w+\*?\s+(bolt_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2509_01742_b300 import bolt as B
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(B._lib, name), name
    assert sorted(B.EXPORTED) == names


def test_strerror_and_codes():
    from paper_2509_01742_b300 import bolt as B
    assert B.bolt_strerror(B.BOLT_OK) == b"ok"
    assert b"poisoned" in B.bolt_strerror(B.BOLT_E_OVERFLOW)
    assert (B.BOLT_E_ARG, B.BOLT_E_NOMEM, B.BOLT_E_OVERFLOW, B.BOLT_E_STATE, B.BOLT_E_DUPKEY) == \
        (O.E_ARG, O.E_NOMEM, O.E_OVERFLOW, O.E_STATE, O.E_DUPKEY)
    # a page that fails its tag (BOLT_PARAM_INTEGRITY) has the oracle's code too
    assert B.BOLT_E_INTEGRITY == O.E_INTEGRITY
    assert b"integrity" in B.bolt_strerror(B.BOLT_E_INTEGRITY)
    assert B.BOLT_PARAM_INTEGRITY == 14
    assert B.BOLT_PARAM_ROUNDS_PRF == 15


@pytest.mark.parametrize("N,vb,alpha,c", [
    (1 << 16, 8, 0.2, 8), (1 << 24, 56, 0.2, 8), (1 << 28, 24, 0.2, 8), (1 << 30, 56, 0.1, 8),
    (10**6, 8, 0.2, 8), (1 << 20, 8, 0.01, 16), (1 << 12, 24, 0.0, 8), (64, 8, 0.5, 8)])
def test_planner_matches_oracle(N, vb, alpha, c):
    from paper_2509_01742_b300 import bolt as B
    assert B.plan(N, vb, alpha=alpha, c=c) == O.sizing(N, c, alpha, vb)


def test_plan_limits_against_oracle():
    """The planner takes every sizing the oracle takes that fits the device
    layout, with the same derived sizes, and rejects the rest: c above 32;
    lmax = c + ceil(log2 log2 N) + 1 above 32 (the kernels give each page slot
    a warp lane); a value store of 2^29 slots or more (29-bit slot pointers in
    a position-map entry); 2^32 position-map slots or more.  The oracle
    itself accepts lmax up to 64 and has none of the other limits."""
    from paper_2509_01742_b300 import bolt as B
    for log_n in (6, 10, 16, 17, 20, 24, 28, 31):
        N = 1 << log_n
        for c in (1, 2, 8, 16, 24, 25, 26, 27, 28, 30, 32, 33, 40):
            theirs = O.sizing(N, c, 0.2, 8)
            try:
                mine = B.plan(N, 8, alpha=0.2, c=c)
            except B.BoltError as e:
                assert e.rc == B.BOLT_E_ARG
                assert c > 32 or theirs["lmax"] > 32 or theirs["vs_cap"] >= 1 << 29 or \
                    theirs["rows"] * theirs["R"] >= 1 << 32, (N, c)
                continue
            assert c <= 32 and theirs["lmax"] <= 32 and theirs["vs_cap"] < 1 << 29
            assert mine == theirs, (N, c)


def test_budget_policy_matches_oracle():
    from paper_2509_01742_b300 import bolt as B
    # the configured budgets: 2 GB at N=2^24 (56 B values), 16 GB at N=2^30
    assert B.plan(1 << 24, 56, hbm_budget=2 * 10**9)["alpha"] == 0.2
    assert B.plan(1 << 30, 56, hbm_budget=16 * 10**9)["alpha"] == 0.1
    for budget in (10**5, 10**6, 10**7, 10**9):
        try:
            mine = B.plan(1 << 20, 8, hbm_budget=budget)
        except B.BoltError as e:
            assert e.rc == B.BOLT_E_NOMEM
            mine = None
        o = O.OracleMap.__new__(O.OracleMap)
        try:
            O.OracleMap.__init__(o, 1 << 20, 8, hbm_budget=budget)
            theirs = o.info()
            o.close()
        except O.OracleError:
            theirs = None
        assert mine == theirs


def test_bad_arguments_rejected_on_host():
    from paper_2509_01742_b300 import bolt as B
    for args in [(32, 8), (1 << 16, 12), (1 << 16, 0), (1 << 16, 512)]:
        with pytest.raises(B.BoltError):
            B.plan(*args)
    for kb in (0, 2, 5, 16):
        with pytest.raises(B.BoltError):
            B.plan(1 << 16, 8, key_bytes=kb)


def test_four_byte_keys_plan_like_eight_byte_keys():
    """A map of 4-byte keys holds them zero-extended: the same sizing, pages
    and records as 8-byte keys, only the reported key width differs."""
    from paper_2509_01742_b300 import bolt as B
    for N, vb in [(10**6, 8), (1 << 20, 24)]:
        four, eight = B.plan(N, vb, key_bytes=4), B.plan(N, vb, key_bytes=8)
        assert four["key_bytes"] == 4 and eight["key_bytes"] == 8
        four.pop("key_bytes"), eight.pop("key_bytes")
        assert four == eight


def test_binding_layouts_match_header(tmp_path):
    """Every struct the binding mirrors has the size and field offsets that a C
    compiler gives the header's declaration, and every #define constant the
    binding repeats has the header's value."""
    import ctypes
    import subprocess
    from paper_2509_01742_b300 import bolt as B
    structs = ["bolt_info_t", "bolt_stats_t", "bolt_profile_t", "bolt_tune_t", "bolt_image_t",
               "bolt_req_info_t", "bolt_server_stats_t"]
    lines = ['#include <stdio.h>', '#include "bolt.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for name, _ in getattr(B, s)._fields_:
            lines.append(f'printf("{s}.{name} %zu\\n", offsetof({s}, {name}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-include",
                    "stddef.h", str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], check=True, capture_output=True,
                              text=True).stdout.split("\n") if line)
    for s in structs:
        cls = getattr(B, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert int(got[f"{s}.{name}"]) == getattr(cls, name).offset, f"{s}.{name}"
    text = open(os.path.join(ROOT, "include", "bolt.h")).read()
    defines = dict(re.findall(r"#define\s+(BOLT_\w+)\s+(-?\d+)", text))
    assert defines, "no numeric #define found"
    for name, value in defines.items():
        if hasattr(B, name):
            assert getattr(B, name) == int(value), name
    assert int(defines["BOLT_PROF_CLASSES"]) == len(B.PROF_NAMES)
