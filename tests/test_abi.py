"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/*.h declares.
No GPU needed (no compute call is made)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(tpmg_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_1402_3545_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1402_3545_gb300 import tpmg
    assert set(declared_symbols()) <= set(tpmg.exported_symbols()) | {"tpmg_nn_create"}


def test_status_strings_without_gpu():
    from paper_1402_3545_gb300 import tpmg
    lib = tpmg.load()
    assert lib.tpmg_status_string(0) == b"ok"
    assert lib.tpmg_status_string(4) == b"not converged"


def test_grid_argument_checks_without_gpu():
    """Grid creation is pure host logic: divisibility and size checks, level rule."""
    from paper_1402_3545_gb300 import tpmg
    g = tpmg.create_grid(512, 512, 128, 0)
    assert tpmg.grid_nlevels(g) == 7
    assert tpmg.grid_level_size(g, 1) == (8, 8)
    tpmg.destroy_grid(g)
    g = tpmg.create_grid(64, 64, 64, 0)
    assert tpmg.grid_nlevels(g) == 4
    tpmg.destroy_grid(g)
    g = tpmg.create_grid(256, 128, 32, 0)
    assert tpmg.grid_nlevels(g) == 6 and tpmg.grid_level_size(g, 1) == (8, 4)
    tpmg.destroy_grid(g)
    import pytest
    with pytest.raises(tpmg.TpmgError):
        tpmg.create_grid(60, 64, 8, 4)  # 60 not divisible by 8
    with pytest.raises(tpmg.TpmgError):
        tpmg.create_grid(64, 64, 300, 0)  # nz above the supported maximum


def test_default_params_layout_without_gpu():
    """tpmg_default_params fills every field of the binding's struct: a field missing or out of
    place in the binding would show up as a wrong default here."""
    import pytest
    from paper_1402_3545_gb300 import tpmg
    p = tpmg.default_params()
    assert (p.nu_pre, p.nu_post, p.n_coarse, p.max_iter) == (2, 2, 2, 100)
    assert (p.rho, p.tol, p.prec, p.use_graph, p.timeout_s, p.zero_guess, p.coarse_bf16) == (0.8, 1e-6, tpmg.DW, 1, 1.0,
                                                                                           0, 0)
    with pytest.raises(TypeError):
        tpmg.default_params(zero_gues=1)


def test_solve_memory_reference_model():
    """The whole-solve byte model bench.py reports: per V(2,2) cycle and fine cell
    17.25 + 20.25 * sum_{j=1}^{L-2} 4^-j + 9 * 4^-(L-1) memory references of the paper's kernels
    (about 23.7 for four levels, 24.0 for seven), plus one Smooth (3) per solve."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_model", os.path.join(os.path.dirname(__file__), "..", "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for L, nx, nz in [(4, 64, 64), (7, 512, 128)]:
        cells = [0] + [(nx >> (L - l)) ** 2 * nz for l in range(1, L + 1)]
        closed = 17.25 + 20.25 * sum(4.0 ** -j for j in range(1, L - 1)) + 9 * 4.0 ** -(L - 1)
        for iters in (1, 6):
            got = bench.solve_memrefs(cells, iters) / cells[L]
            assert abs(got - (3 + iters * closed)) < 1e-12
    assert abs(closed - 23.9956) < 1e-4


def test_set_allocator_argument_checks_without_gpu():
    from paper_1402_3545_gb300 import tpmg
    lib = tpmg.load()
    alloc = tpmg.ALLOC_FN(lambda n, c: None)
    assert lib.tpmg_set_allocator(alloc, tpmg.FREE_FN(), None) == tpmg.ERR_ARG
    assert b"both" in lib.tpmg_last_error()
    assert lib.tpmg_set_allocator(tpmg.ALLOC_FN(), tpmg.FREE_FN(), None) == tpmg.OK


def test_header_is_plain_c(tmp_path):
    """include/tpmg.h is a C ABI: it compiles as strict C99 (no C++ or CUDA types in the signatures)
    and every declared function can be referenced from C."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        import pytest
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    refs = "\n".join(f"    (void)&{n};" for n in declared_symbols())
    src.write_text('#include "tpmg.h"\nint main(void) {\n' + refs + "\n    return 0;\n}\n")
    res = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                          "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def _kernel_table():
    rows = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "kernel_table.txt")):
        if line.strip() and not line.startswith("#"):
            name, fl, mem, memc = line.split()
            rows[name] = (float(fl), float(mem), float(memc))
    return rows


def test_cycle_accounting_reproduces_the_papers_kernel_table():
    """bench.py's cycle accounting (which kernels run on which level, weighted by the level's cells)
    fed with the paper's per-kernel counts reproduces the paper's totals for its V(1,1) on 5 levels
    (Sec. 4.1, Table KernelTable): MemC 29.6 per fine cell (23 on the fine level), Mem 67.2 and
    FLOPs 149.4 given the table's fine-level rows; and the fused CG's sums."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_model2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    t = _kernel_table()
    cells = [0] + [4.0 ** (l - 5) for l in range(1, 6)]  # fine level = 1; each coarser level 1/4
    for col in (0, 1, 2):
        k = {name: t[name][col] for name in ("Smooth", "ResSmooth", "Res", "Prolongate", "ResNorm")}
        kw = dict(nu_pre=1, nu_post=1, n_coarse=2, smooth=k["Smooth"], residual=k["Res"],
                  restrict_smooth=k["ResSmooth"], prolongate=k["Prolongate"], norm=k["ResNorm"])
        fine = bench.cycle_memrefs(cells, fine_only=True, **kw)
        total = bench.cycle_memrefs(cells, **kw)
        if col == 2:
            # MemC: the fine level is the sum of its kernels
            assert fine == t["FineLevelOnly"][2]
        # the coarser levels on top of the table's fine-level row give the table's total
        coarse = total - fine
        assert abs(t["FineLevelOnly"][col] + coarse - t["Total"][col]) < 0.05, (col, coarse)
    assert t["SpMV"][2] + t["Tridiag"][2] == t["CGTotal"][2]
    assert t["SpMV"][0] + t["Tridiag"][0] == t["CGTotal"][0]


def test_binding_refuses_host_tensors_without_gpu():
    """No CPU fallback: every field argument must be a CUDA tensor of the precision's dtype and size;
    host tensors are refused before the library is called (here without a GPU)."""
    import pytest
    import torch
    from paper_1402_3545_gb300 import tpmg
    x = torch.zeros(4 * 4 * 2, dtype=torch.float64)
    with pytest.raises(TypeError, match="CUDA tensor"):
        tpmg.apply_A(0, 1, tpmg.F64, x, x, x.numel())
    with pytest.raises(TypeError, match="CUDA tensor"):
        tpmg.residual_restrict_smooth(0, 1, tpmg.DW, 0.8, x, x, x, x, x.numel(), x.numel())
    with pytest.raises(TypeError, match="CUDA tensor"):
        tpmg.mg_solve(0, tpmg.default_params(prec=tpmg.F64), x, x, x.numel())
    with pytest.raises(TypeError, match="scalar outputs"):
        tpmg._scalar_out(torch.zeros(1, dtype=torch.float64))
    # page-locked host fields are accepted only by the double-word and mixed solves
    with pytest.raises(ValueError, match="prec DW or MIXED"):
        tpmg.mg_solve_mapped(0, tpmg.default_params(prec=tpmg.F64), x, x, x.numel())
