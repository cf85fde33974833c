"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/mpr.h declares; the ctypes structures match the C layout.
No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2212_01317_gb300 import mpr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpr3?_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_bound_names():
    decl = declared_functions()
    assert "mpr_create" in decl and "mpr_simulate" in decl and "mpr_predict" in decl
    assert sorted(mpr.EXPORTS) == decl


def test_library_exports_every_declared_symbol():
    lib = mpr.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", mpr._build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (mpr3?_\w+)", out))
    assert set(declared_functions()) <= exported


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "mpr.h"
#define O(T, f) printf(#T "." #f " %zu\\n", offsetof(T, f))
int main(void) {
  printf("mpr_grid %zu\\nmpr_options %zu\\nmpr_info %zu\\n", sizeof(mpr_grid),
         sizeof(mpr_options), sizeof(mpr_info));
  printf("mpr_grid3 %zu\\nmpr3_info %zu\\nmpr_tuning %zu\\nmpr_profile %zu\\n",
         sizeof(mpr_grid3), sizeof(mpr3_info), sizeof(mpr_tuning), sizeof(mpr_profile));
  O(mpr_options, cal_method); O(mpr_options, t_init); O(mpr_options, sim_graph);
  O(mpr_options, cal_points); O(mpr_options, sim_tail); O(mpr_options, sweep_form);
  O(mpr_options, pair_tail); O(mpr_options, sweep_form_bulk); O(mpr_options, stop_rule);
  O(mpr_options, n_fit); O(mpr_options, n_f);
  O(mpr_tuning, trial_ms);
  O(mpr_info, n_slices); O(mpr3_info, n_gap); O(mpr3_info, cal_gap_updates);
  O(mpr_tuning, ms); O(mpr_profile, sim_tail_updates); O(mpr_profile, sim_tail_ms);
  O(mpr_options, seed); O(mpr_options, slice_id); O(mpr_options, t_lo);
  O(mpr_options, group); O(mpr_options, cuda_stream);
  O(mpr_info, n_gap); O(mpr_info, zmin); O(mpr_info, realizations); O(mpr_info, batch);
  O(mpr_info, gap_updates); O(mpr_info, device_bytes);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True,
                                                        text=True).stdout.split("\n") if l)
    assert int(got["mpr_grid"]) == ctypes.sizeof(mpr.mpr_grid)
    assert int(got["mpr_options"]) == ctypes.sizeof(mpr.mpr_options)
    assert int(got["mpr_info"]) == ctypes.sizeof(mpr.mpr_info)
    for T in ("mpr_grid3", "mpr3_info", "mpr_tuning", "mpr_profile"):
        assert int(got[T]) == ctypes.sizeof(getattr(mpr, T)), T
    for k, v in got.items():
        if "." in k:
            T, f = k.split(".")
            assert getattr(getattr(mpr, T), f).offset == int(v), k


def test_default_options_without_gpu():
    o = mpr.mpr_default_options()
    assert (o.q, o.J, o.n_max, o.n_eq, o.n_meas, o.n_bisect) == (0.5, 1.0, 200, 25, 20, 24)
    assert o.t_hi == 2.0 and abs(o.t_lo - 1e-4) < 1e-9 and o.overrelax == 1
    assert o.sweep_form == -1 and o.sim_tail == 0 and o.cal_points == 1 and o.pair_tail == 4096
    assert (o.sweep_form_bulk, o.stop_rule, o.n_fit, o.n_f) == (-1, 0, 20, 5)
    assert mpr.load().mpr_status_string(4) == b"no sample pair"
    with pytest.raises(TypeError):
        mpr.mpr_default_options(nonsense=1)
