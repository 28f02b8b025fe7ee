"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/sisdc.h (no compute calls here)."""
import ctypes
import os

import pytest

from paper_2504_18526_gb300 import sisdc


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(sisdc.LIB_PATH):
        from paper_2504_18526_gb300.build import build
        build()
    return sisdc.load()


def test_exports_every_declared_symbol(lib):
    names = sisdc.header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    """sizeof/offsetof of the header's structs, compiled by the C compiler,
    equal the binding's ctypes layouts."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sisdc.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu ", sizeof(sisdc_level_desc),'
        ' sizeof(sisdc_problem), sizeof(sisdc_stats), offsetof(sisdc_level_desc, lo),'
        ' offsetof(sisdc_problem, cg_rtol), offsetof(sisdc_stats, launches),'
        ' sizeof(sisdc_ens_instance), offsetof(sisdc_ens_instance, dt), sizeof(sisdc_ens_opts),'
        ' offsetof(sisdc_ens_opts, cg_rtol)); printf("%zu %zu\\n", sizeof(sisdc_stab_opts),'
        ' offsetof(sisdc_stab_opts, fmg_cycles)); return 0;}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(sisdc.sisdc_level_desc), ctypes.sizeof(sisdc.sisdc_problem),
                    ctypes.sizeof(sisdc.sisdc_stats), sisdc.sisdc_level_desc.lo.offset,
                    sisdc.sisdc_problem.cg_rtol.offset, sisdc.sisdc_stats.launches.offset,
                    ctypes.sizeof(sisdc.sisdc_ens_instance), sisdc.sisdc_ens_instance.dt.offset,
                    ctypes.sizeof(sisdc.sisdc_ens_opts), sisdc.sisdc_ens_opts.cg_rtol.offset,
                    ctypes.sizeof(sisdc.sisdc_stab_opts), sisdc.sisdc_stab_opts.fmg_cycles.offset]


def test_invalid_problem_rejected_without_gpu(lib):
    p = sisdc.make_problem({"pde": "burgers", "ncomp": 3, "nu": 1e-3, "dim": 2})
    with pytest.raises(sisdc.SisdcError) as ei:
        sisdc.sisdc_create(p)
    assert ei.value.status == sisdc.SISDC_E_ARG


def test_invalid_ensemble_rejected_without_gpu(lib):
    good = dict(nel=(4, 4), P=3, nu=1e-3, adv=(1.0, 0.0), dt=1e-3)
    for bad in (dict(good, P=9), dict(good, P=1), dict(good, dt=0.0), dict(good, nel=(0, 4)),
                dict(good, nu=-1.0), dict(good, adv=(float("nan"), 0.0))):
        with pytest.raises(sisdc.SisdcError) as ei:
            sisdc.sisdc_ens_create([sisdc.make_ens_instance(bad)], sisdc.make_ens_opts())
        assert ei.value.status == sisdc.SISDC_E_ARG
    for opts in (sisdc.make_ens_opts(M=9), sisdc.make_ens_opts(Mc=6), sisdc.make_ens_opts(start="fmg1"),
                 sisdc.make_ens_opts(si_stages=3), sisdc.make_ens_opts(cg_rtol=0.0)):
        with pytest.raises(sisdc.SisdcError) as ei:
            sisdc.sisdc_ens_create([sisdc.make_ens_instance(good)], opts)
        assert ei.value.status == sisdc.SISDC_E_ARG


def test_set_allocator_rejects_without_gpu(lib):
    """sisdc_set_allocator checks its arguments before touching the device:
    a NULL context, or alloc without release, is SISDC_E_ARG."""
    assert lib.sisdc_set_allocator(None, sisdc.ALLOC_FN(), sisdc.RELEASE_FN(), None) == sisdc.SISDC_E_ARG
    dummy_alloc = sisdc.ALLOC_FN(lambda n, s, u: None)
    assert lib.sisdc_set_allocator(None, dummy_alloc, sisdc.RELEASE_FN(), None) == sisdc.SISDC_E_ARG
