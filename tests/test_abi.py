"""C-ABI library checks that need no GPU: it loads, exports every symbol the
header declares, and its host-only functions agree with their definitions."""
import ctypes as C
import subprocess

import pytest

from oracle import lra_oracle as O


@pytest.fixture(scope="module")
def lra():
    import paper_1607_02925_gb300 as m
    return m


def test_library_exports_every_declared_symbol(lra):
    declared = lra.declared_symbols()
    assert len(declared) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", lra.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(lra.lib, s)


def test_stream_key_matches_definition(lra):
    for seed, st, a, b in [(0, 1, 0, 0), (7, 4, 3, 11), (2**64 - 1, 5, 2**40, 9)]:
        assert lra.lra_stream_key(seed, st, a, b) == O.stream_key(seed, st, a, b)


def test_options_defaults_and_status_names(lra):
    o = lra.options()
    assert o.struct_size == C.sizeof(lra.LraOptions)
    assert (o.shift_policy, o.theta_eta, o.theta_m, o.max_epochs, o.max_outer) == (0, 0.25, 2.0, 60, 2000)
    assert lra.lra_status_str(0) == "LRA_OK"
    assert lra.lra_status_str(11) == "LRA_EUNSUPPORTED"
    # the accelerated and partitioned options default off, with the oracle's parameters
    from oracle import lra_oracle as O
    from oracle import lra_partition as P
    oo = O.Options()
    assert (o.acc, o.acc_theta, o.acc_max_outer, o.acc_target) == (0, oo.acc_theta, oo.acc_max_outer,
                                                                    oo.acc_target)
    assert (o.partition, o.part_max_iters) == (0, 2000)
    assert P.adaptive_solve.__defaults__[-1] == o.part_max_iters
    assert (lra.LRA_STREAM_PART, lra.LRA_STREAM_BLOCK) == (P.STREAM_PART, P.STREAM_BLOCK)


def test_struct_layouts_match_header(lra):
    # sizes of the C structs as laid out by the C compiler
    src = r'''
    #include <stdio.h>
    #include "lra.h"
    int main(void) { printf("%zu %zu %zu\n", sizeof(lra_options), sizeof(lra_report), sizeof(lra_solve_info)); return 0; }
    '''
    import os
    import tempfile
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(td, "s")
        subprocess.run(["gcc", "-I", os.path.join(root, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [C.sizeof(lra.LraOptions), C.sizeof(lra.LraReport), C.sizeof(lra.LraSolveInfo)]


def test_invalid_arguments_rejected_without_gpu(lra):
    # null pointers are rejected before any device work
    assert lra.lib.lra_init(0, 0, None) == 1
    assert lra.lib.lra_solve(None, 1, 2, 1e-3, 0, None, None, None, None) == 1
