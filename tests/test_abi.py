"""The C ABI library loads and exports every entry point include/hikf.h declares."""
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def _declared():
    text = (ROOT / "include" / "hikf.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hikf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1404_3816_gb300 import binding, build
    if not binding.LIB_PATH.exists():
        build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hikf_create", "hikf_assimilate", "hikf_get_mean", "hikf_get_variance", "hikf_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in _declared() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1404_3816_gb300 import binding
    assert sorted(binding.EXPORTED) == _declared()


def test_options_default_without_gpu(lib):
    from paper_1404_3816_gb300 import binding
    o = binding.options()
    assert o.cheb_order == 8 and o.leaf_size == 64 and o.max_depth == -1 and o.precision == 0


def test_release_cached_memory_without_a_pool(lib):
    # the library's pool is made on the first device allocation; with none made, releasing
    # the cache is a no-op that needs no device
    from paper_1404_3816_gb300 import binding
    binding.release_cached_memory()


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    import numpy as np
    from paper_1404_3816_gb300 import binding, workload as W
    w = W.small(grid=(10, 8), n=4, seed=1)
    good = dict(points=w.points, q=w.q, h_rowptr=w.h_rowptr, h_col=w.h_col, h_val=w.h_val, r_diag=w.r_diag)
    bad_cases = [
        dict(r_diag=np.zeros(w.n)),
        dict(h_col=np.where(np.arange(w.nnz) == 0, w.m + 5, w.h_col)),
        dict(q=W.KernelSpec(5, 0.01, 8.0)),             # no such family
        dict(q=W.KernelSpec(W.WHITE, 0.01, 8.0)),      # the white kernel is for P_0 only
        dict(q=W.KernelSpec(W.LOG, 0.01, 8.0, 0.5)),   # a generalised covariance: H^2 product only
        dict(q=W.KernelSpec(W.GCF, 0.01, 8.0, 2.5)),   # GCF exponent beyond (0, 2]
        dict(q=W.KernelSpec(W.GCF, 0.01, 8.0, 0.0)),
        dict(p0=W.KernelSpec(5, 1.0, 8.0)),
        dict(p0=W.KernelSpec(W.LOG, 1.0, 8.0, 0.5)),
        dict(q=W.KernelSpec(1, -1.0, 8.0)),
        dict(points=np.where(np.arange(w.m * 2).reshape(w.m, 2) == 3, np.nan, w.points)),
    ]
    for bad in bad_cases:
        kw = dict(good)
        kw.update(bad)
        with pytest.raises(binding.HikfError) as e:
            binding.Filter(**kw)
        assert e.value.code == binding.HIKF_EINVAL
    with pytest.raises(binding.HikfError):
        binding.Filter(**good, cheb_order=40)
    # a full R that is not symmetric or not finite is refused on the host
    bad_r = np.eye(w.n) * 1e-3
    bad_r[0, 1] = 1e-4
    for r_full in (bad_r, np.full((w.n, w.n), np.nan)):
        kw = dict(good)
        kw.pop("r_diag")
        with pytest.raises(binding.HikfError) as e:
            binding.Filter(**kw, r_diag=None, r_full=r_full)
        assert e.value.code == binding.HIKF_EINVAL


def test_serving_schedule_and_footprint_without_gpu():
    from paper_1404_3816_gb300 import serve
    streams = serve.serving_streams(count=64)
    sides = [w.grid[0] for w in streams]
    assert min(sides) >= 64 and max(sides) <= 1024
    assert {w.n for w in streams} <= {16, 32, 64, 128, 256}
    sched = serve.poisson_schedule(streams, rate=500.0, seconds=2.0)
    assert 800 < len(sched) < 1200                     # ~ rate x seconds
    assert all(0 <= s < 64 for _, s in sched)
    big = max(streams, key=lambda w: w.m)
    assert serve.footprint_bytes(big) > 2 * big.m * 4 * ((big.n + 31) // 32 * 32)


_CTYPES = {"int": "c_int", "double": "c_double", "int64_t": "c_int64", "void*": "c_void_p"}


def _header_structs():
    """{typedef name: [(C type, field name), ...]} of the plain structs in include/hikf.h."""
    text = (ROOT / "include" / "hikf.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"([A-Za-z_][\w ]*?\s*\*?)\s*(\w+)$", decl)
            assert m, decl
            fields.append((m.group(1).replace(" ", ""), m.group(2)))
        out[name] = fields
    return out


@pytest.mark.parametrize("cname,pyname", [("hikf_kernel", "Kernel"), ("hikf_options", "Options"),
                                          ("hikf_info_t", "Info")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors of the ABI structs have the header's fields, in order, with the
    same C types (a mismatch would shift every later field)."""
    import ctypes as C
    from paper_1404_3816_gb300 import binding
    header = _header_structs()[cname]
    mirror = getattr(binding, pyname)._fields_
    assert [f for _, f in header] == [f for f, _ in mirror]
    for (ctype, field), (_, pytype) in zip(header, mirror):
        assert pytype is getattr(C, _CTYPES[ctype]), (cname, field, ctype, pytype)


def _cc():
    import shutil
    return shutil.which("gcc") or shutil.which("cc")


def test_header_is_plain_c(tmp_path):
    """include/hikf.h compiles as C99 on its own (no C++ or CUDA types in the boundary)."""
    import subprocess
    cc = _cc()
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "hikf.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", str(ROOT / "include"),
                        "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_the_library(tmp_path, lib):
    """A C program links against libhikf.so and calls host-only entry points: the
    defaults, the rejection of a NULL argument with HIKF_EINVAL, hikf_step of no handle."""
    import subprocess
    from paper_1404_3816_gb300 import binding
    cc = _cc()
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(
        '#include <stdio.h>\n#include "hikf.h"\n'
        "int main(void) {\n"
        "  hikf_options o;\n"
        "  if (hikf_options_default(&o) != HIKF_OK) return 1;\n"
        "  if (hikf_options_default(NULL) != HIKF_EINVAL) return 2;\n"
        "  if (hikf_step(NULL) != -1) return 3;\n"
        '  printf("%d %d %d %d %d %d\\n", o.cheb_order, o.leaf_size, o.max_depth, o.precision, o.graph, o.m2l);\n'
        "  return 0;\n}\n")
    exe = tmp_path / "use"
    libdir = binding.LIB_PATH.parent
    r = subprocess.run([cc, "-std=c99", "-I", str(ROOT / "include"), str(src), "-o", str(exe), "-L", str(libdir),
                        "-lhikf", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.split() == ["8", "64", "-1", "0", "1", "0"]


def test_batch_rejects_bad_arguments_without_device_work(lib):
    import ctypes as C
    from paper_1404_3816_gb300 import binding
    assert lib.hikf_assimilate_batch(None, None, -1) == binding.HIKF_EINVAL
    assert b"count" in lib.hikf_last_error(None)
    assert lib.hikf_assimilate_batch(None, None, 0) == binding.HIKF_OK      # an empty batch
    assert lib.hikf_assimilate_batch(None, None, 2) == binding.HIKF_EINVAL
    hs = (C.c_void_p * 2)(None, None)
    ys = (C.c_void_p * 2)(None, None)
    assert lib.hikf_assimilate_batch(hs, ys, 2) == binding.HIKF_EINVAL     # a NULL handle
    assert b"NULL" in lib.hikf_last_error(None)
    with pytest.raises(binding.HikfError) as e:
        binding.assimilate_batch([object()], [])
    assert e.value.code == binding.HIKF_EINVAL


def test_sweep_products_option_is_checked_without_gpu(lib):
    from paper_1404_3816_gb300 import binding, workload as W
    w = W.small(grid=(10, 8), n=4, seed=1)
    for bad in (1, 3, 6, -4):
        with pytest.raises(binding.HikfError) as e:
            binding.Filter.from_workload(w, precision="mixed", sweep_products=bad)
        assert e.value.code == binding.HIKF_EINVAL and "sweep_products" in str(e.value)
