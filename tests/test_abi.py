"""CPU-side checks of the C ABI: the library builds, loads and exports every
declared symbol; host-side planning and argument validation need no GPU."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_0911_5631_gb300 as md
from paper_0911_5631_gb300 import build as mdbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RC = md.WCA_RC


@pytest.fixture(scope="module")
def libmd():
    mdbuild.build()
    return md.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "md.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(libmd):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(libmd, n), n
    # and the binding covers exactly the declared set
    assert sorted(s[0] for s in md.SIGNATURES) == names


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(md, "_lib", None)
    monkeypatch.setattr(md, "LIB_PATH", "/nonexistent/libmd.so")
    with pytest.raises(md.MDLibraryMissing):
        md.lib()


def test_struct_layouts_match_header(tmp_path):
    # compile a probe against include/md.h and compare sizes and offsets
    import ctypes as C
    import subprocess
    structs = [md.md_params, md.md_plan_t, md.md_measure_t, md.md_kernel_stats_t, md.md_replica_desc]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "md.h"', 'int main(void) {']
    for s in structs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % s.__name__)
        for f, _ in s._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (s.__name__, f))
    lines.append("return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = []
    for s in structs:
        want.append(C.sizeof(s))
        want += [getattr(s, f).offset for f, _ in s._fields_]
    assert got == want


@pytest.mark.parametrize("n,rho,skin,even", [(2048, 0.8, 0.0, False), (1048576, 0.8, 0.4, False),
                                              (8388608, 0.6, 0.4, False), (8388608, 1.0, 0.4, False),
                                              (110592, 0.8, 0.4, True), (110592, 0.8, 0.6, True)])
def test_plan_matches_oracle_grid(libmd, n, rho, skin, even):
    L = (n / rho) ** (1.0 / 3.0)
    p = md.md_default_params()
    p.even_cells = int(even)
    plan = md.md_plan([L] * 3, n, RC, skin, 0.005, p)
    G, ok = oracle.cell_grid([L] * 3, RC + skin, even=even)
    assert ok
    assert list(plan.G) == list(G)
    assert plan.n_cells == int(np.prod(G))
    assert plan.ushift == 1.0
    assert plan.nbr_capacity >= 16


def test_plan_paper_cell_counts(libmd):
    # Table 5, delta = 0.4: 32768 cells with the even rounding
    L = 48 / 0.8 ** (1.0 / 3.0)
    p = md.md_default_params()
    p.even_cells = 1
    assert md.md_plan([L] * 3, 48 ** 3, RC, 0.4, 0.005, p).n_cells == 32768


@pytest.mark.parametrize("kw", [dict(n=0), dict(n=-5), dict(rc=0.0), dict(skin=-0.1), dict(dt=0.0),
                                dict(box=[3.0, 20.0, 20.0]), dict(n=1 << 26), dict(box=[float("nan")] * 3)])
def test_plan_rejects_bad_arguments(libmd, kw):
    args = dict(box=[20.0] * 3, n=1000, rc=RC, skin=0.4, dt=0.005)
    args.update(kw)
    with pytest.raises(md.MDError) as e:
        md.md_plan(args["box"], args["n"], args["rc"], args["skin"], args["dt"])
    assert e.value.code == md.MD_EINVAL


def test_cell_list_only_requires_zero_skin(libmd):
    p = md.md_default_params()
    p.cell_list_only = 1
    with pytest.raises(md.MDError):
        md.md_plan([20.0] * 3, 1000, RC, 0.4, 0.005, p)
    assert md.md_plan([20.0] * 3, 1000, RC, 0.0, 0.005, p).nbr_capacity == 0


def test_ushift_rule(libmd):
    assert md.md_plan([30.0] * 3, 1000, 2.5, 0.3, 0.005).ushift == 0.0
    p = md.md_default_params()
    p.ushift = 0.25
    assert md.md_plan([30.0] * 3, 1000, 2.5, 0.3, 0.005, p).ushift == 0.25
    assert oracle.wca_shift(RC) == 1.0 and oracle.wca_shift(2.5) == 0.0


def test_default_params(libmd):
    p = md.md_default_params()
    assert p.precision == md.MD_PREC_MIXED and p.reorder_interval == 100 and p.use_graphs == 1
    assert np.isnan(p.ushift) and p.device == -1 and p.shell_bins == 1


def test_plan_bytes_include_the_shell_bin_counts(libmd):
    # 7 planes of one byte per atom hold the entry counts below the shell-bin
    # boundaries; they are part of the device footprint in both forms
    box = [20.0] * 3
    for prec in (md.MD_PREC_MIXED, md.MD_PREC_FP64):
        p = md.md_default_params()
        p.precision = prec
        p.nbr_capacity = 48
        # powers of two: the pair buffers hold n rounded up to one
        b1 = md.md_plan(box, 4096, md.WCA_RC, 0.4, 0.005, p).device_bytes
        b2 = md.md_plan(box, 8192, md.WCA_RC, 0.4, 0.005, p).device_bytes
        per_atom = (b2 - b1) / 4096
        real = 8 if prec == md.MD_PREC_FP64 else 4
        pos4 = 32 if prec == md.MD_PREC_FP64 else 16
        state = 3 * 4 + 3 * real + 24 + 3 * real + 3 * real + 2 * pos4 + 16 + 8 + 3 * real + 24 + 3 * real
        # order, nn, lim, io, list; the per-block energy partials add 24 B
        # per 256 atoms
        assert per_atom == pytest.approx(state + 4 + 4 + 7 + 48 + 48 * 4 + 24 / 256, abs=0.01)
        # between powers of two the two pair buffers are padded to the next
        # one (the list columns and energy partials round up by a few KB)
        b3 = md.md_plan(box, 5000, md.WCA_RC, 0.4, 0.005, p).device_bytes
        assert b3 - (b1 + per_atom * 904) == pytest.approx(2 * pos4 * (8192 - 5000), abs=5000)


def test_ensemble_replica_bytes_needs_no_gpu(libmd):
    small = md.replica_desc([8.0] * 3, 410)
    big = md.replica_desc([32.0] * 3, 26214)
    b0, b1 = md.md_ensemble_replica_bytes(small), md.md_ensemble_replica_bytes(big)
    assert 0 < b0 < b1
    # roughly the per-atom state plus the list: a few hundred bytes per atom
    assert 150 * 26214 < b1 < 2000 * 26214
    bad = md.replica_desc([8.0] * 3, 410)
    bad.reserved[0] = 1
    assert md.md_ensemble_replica_bytes(bad) == 0
    assert md.md_ensemble_replica_bytes(md.replica_desc([8.0] * 3, 410, skin=0.0)) == 0  # list form only
    assert md.md_ensemble_replica_bytes(md.replica_desc([4.0] * 3, 50)) == 0  # fewer than 3 cells


def test_kernel_variants_and_builds_are_validated(libmd):
    # the ablation variants exist for the mixed form with a neighbour list;
    # one flag at a time; the build selector takes its three values
    def plan(**kw):
        p = md.md_default_params()
        skin = 0.0 if kw.get("cell_list_only") else 0.4
        for k, v in kw.items():
            setattr(p, k, v)
        return md.md_plan([20.0] * 3, 1000, RC, skin, 0.005, p)
    for v in md.VARIANTS.values():
        plan(variant=v)
    for bad in ({"variant": 3}, {"variant": 16}, {"variant": md.MD_VARIANT_LIST_ROWS, "precision": md.MD_PREC_FP64},
                {"variant": md.MD_VARIANT_BLOCK64, "cell_list_only": 1}, {"build_kernel": 3}):
        with pytest.raises(md.MDError) as e:
            plan(**bad)
        assert e.value.code == md.MD_EINVAL
    for b in (md.MD_BUILD_AUTO, md.MD_BUILD_THREAD, md.MD_BUILD_WARP):
        plan(build_kernel=b)
