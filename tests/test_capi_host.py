"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-only helpers agree with the oracle."""

from __future__ import annotations

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_0906_1775_gb300 as mm
    from paper_0906_1775_gb300 import build
    if not os.path.exists(mm.library_path()):
        build.build()
    return mm


def _declared():
    txt = open(os.path.join(ROOT, "include", "madmap.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(madmap_[a-z_A-Z0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    mm = _lib()
    lib = mm.load()
    names = _declared()
    assert "madmap_solve" in names and "madmap_apply_ATNA" in names
    for n in names:
        assert hasattr(lib, n), n
    bound = {p[0] for p in mm._lib.PROTOTYPES}
    assert set(names) == bound, set(names) ^ bound


def test_version_and_error_strings():
    mm = _lib()
    assert mm.load().madmap_version().startswith(b"madmap")
    assert isinstance(mm.madmap_last_error(), str)


@pytest.mark.parametrize("params", [(64, 100.0, 1.0, 0.1, 2.0), (128, 100.0, 1.3, 0.05, 1.2),
                                    (8, 100.0, 0.9, 5.0, 1.5), (4096, 100.0, 1.0, 0.1, 2.0), (12, 180.0, 1.0, 0.03, 1.7)])
def test_noise_filter_matches_oracle(params):
    from oracle.noise import filter_lags
    mm = _lib()
    n, fs, s, fk, a = params
    lib_f, lib_g = mm.noise_filter(n, fs, s, fk, a, with_grad=True)
    ora_f, ora_g = filter_lags(n, fs, s, fk, a, with_grad=True)
    assert np.max(np.abs(lib_f - ora_f)) <= 1e-13 * np.max(np.abs(ora_f))
    assert np.max(np.abs(lib_g - ora_g)) <= 1e-12 * np.max(np.abs(ora_g))


def test_noise_filter_rejects_bad_args():
    mm = _lib()
    with pytest.raises(mm.MadmapError):
        mm.noise_filter(0, 100.0, 1.0, 0.1, 2.0)
    with pytest.raises(mm.MadmapError):
        mm.noise_filter(8, 100.0, -1.0, 0.1, 2.0)


@pytest.mark.parametrize("n_c,longest", [(2 ** 12, 2 ** 18), (2 ** 14, 2 ** 20), (2 ** 15, 648000), (16, 100),
                                          (2 ** 12, 5000), (1, 10)])
def test_paper_fft_length_matches_oracle(n_c, longest):
    from oracle.noise import fft_length
    mm = _lib()
    assert mm.paper_fft_length(n_c, longest) == fft_length(n_c, longest)


def test_noise_filter_vjp_matches_oracle_chain_rule():
    from oracle.noise import filter_lags
    mm = _lib()
    rng = np.random.default_rng(3)
    for params in [(1.0, 0.1, 2.0), (0.8, 0.05, 1.3)]:
        g = rng.standard_normal(64)
        _, dl = filter_lags(64, 100.0, *params, with_grad=True)
        assert np.allclose(mm.madmap_noise_filter_vjp(64, 100.0, *params, g), dl @ g, rtol=1e-11, atol=1e-14)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding marshals has the header's size and field offsets
    (compiled from include/madmap.h by the host C compiler)."""
    import shutil
    import subprocess
    mm = _lib()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    L = mm._lib
    structs = {"madmap_plan_desc": L.madmap_plan_desc, "madmap_plan_stats": L.madmap_plan_stats,
               "madmap_checkpoint": L.madmap_checkpoint, "madmap_solve_opts": L.madmap_solve_opts,
               "madmap_solve_info": L.madmap_solve_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "madmap.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    import ctypes
    seen = 0
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        got = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (name, field, got, value)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    """The C ABI from plain C (no Python, no torch): a program compiled against
    include/madmap.h and linked to libmadmap.so calls the host-side entry points and
    gets argument errors as status codes with a message."""
    import shutil
    import subprocess
    mm = _lib()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = tmp_path / "use.c"
    src.write_text(r'''
#include <stdio.h>
#include "madmap.h"
int main(void) {
  double lags[16], dl[48];
  printf("version %s\n", madmap_version());
  printf("filter %d", (int)madmap_noise_filter(16, 100.0, 1.0, 0.1, 2.0, lags, dl));
  for (int i = 0; i < 16; ++i) printf(" %.17g", lags[i]);
  printf("\n");
  printf("fftlen %lld\n", (long long)madmap_paper_fft_length(1024, 100000));
  madmap_plan_t plan = 0;
  madmap_status st = madmap_plan_create(0, 0, &plan);
  printf("create %d %s\n", (int)st, madmap_last_error());
  st = madmap_noise_filter(0, 100.0, 1.0, 0.1, 2.0, lags, 0);
  printf("badfilter %d\n", (int)st);
  return 0;
}
''')
    lib_dir = os.path.dirname(mm.library_path())
    exe = tmp_path / "use"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", lib_dir,
                    "-lmadmap", "-Wl,-rpath," + lib_dir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    assert out[0].startswith("version madmap")
    f = out[1].split()
    assert f[1] == "0"
    vals = np.array([float(v) for v in f[2:]])
    ref, _ = mm.noise_filter(16, 100.0, 1.0, 0.1, 2.0, with_grad=True)
    assert np.array_equal(vals, ref)
    assert int(out[2].split()[1]) == mm.paper_fft_length(1024, 100000)
    assert out[3].startswith("create -1 ") and len(out[3]) > len("create -1 ")
    assert out[4] == "badfilter -1"


def test_solve_option_defaults():
    """madmap_solve_opts_default (host only): the paper's defaults (50 iterations,
    relative residual 1e-6, Section 5) and the mixed solve's continued refinement."""
    import ctypes
    mm = _lib()
    o = mm._lib.madmap_solve_opts()
    mm.load().madmap_solve_opts_default(ctypes.byref(o))
    assert (o.max_iter, o.rel_tol, o.precision) == (50, 1e-6, mm._lib.MADMAP_FP64)
    assert (o.max_outer, o.inner_rel_tol, o.use_graph, o.iters_per_sync) == (10, 1e-4, 2, 8)
    assert o.refine_precision == mm._lib.MADMAP_DF64
    assert (o.checkpoint_every, o.history_capacity) == (0, 0)
    assert (o.inner_restart, o.final_residual) == (0, 0)
