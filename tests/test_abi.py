"""Host-side checks of the C ABI that need no GPU: the library builds, loads, and
exports every symbol that include/csg.h declares, and the binding agrees with the
header's constants."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "csg.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(csg_[a-z_0-9]+)\s*\(", text)))


def _defines():
    out = {}
    for m in re.finditer(r"#define\s+(CSG_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", open(HEADER).read()):
        out[m.group(1)] = int(m.group(2))
    return out


@pytest.fixture(scope="module")
def lib():
    from paper_1709_03013_gb300 import _build
    return ctypes.CDLL(_build.build())


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1709_03013_gb300 import csg
    assert sorted(csg.EXPORTS) == _declared()


def test_constants_match_header():
    from paper_1709_03013_gb300 import csg
    d = _defines()
    assert d["CSG_OK"] == csg.OK and d["CSG_PENDING"] == csg.PENDING
    assert d["CSG_E_INVAL"] == csg.E_INVAL and d["CSG_E_NOMEM"] == csg.E_NOMEM
    assert d["CSG_E_CUDA"] == csg.E_CUDA and d["CSG_E_TIMEOUT"] == csg.E_TIMEOUT
    assert d["CSG_E_BUSY"] == csg.E_BUSY and d["CSG_E_REJECT"] == csg.E_REJECT
    assert d["CSG_E_NOTFOUND"] == csg.E_NOTFOUND and d["CSG_E_CANCELLED"] == csg.E_CANCELLED
    assert d["CSG_POPC"] == csg.POPC and d["CSG_TC"] == csg.TC
    assert csg.MAX_N == 1 << 18


def test_result_struct_layout():
    from paper_1709_03013_gb300 import csg
    assert ctypes.sizeof(csg._Result) == 88


def test_strerror_and_argument_errors_without_gpu(lib):
    from paper_1709_03013_gb300 import csg
    L = csg.load()
    assert L.csg_strerror(csg.E_INVAL) == b"invalid argument"
    # null context / bad arguments are rejected before any CUDA call
    t = ctypes.c_uint64()
    assert L.csg_serve_submit(None, 2, 10, 0, 0, ctypes.byref(t)) == csg.E_INVAL
    assert L.csg_link(None, None, None) == csg.E_INVAL
    assert L.csg_action(None, None, 0, None, None) == csg.E_INVAL
    assert L.csg_set_info(None, None, None, None, None, None) == csg.E_INVAL


def test_bulk_result_conversion_matches_per_field():
    """The batch calls convert their csg_result arrays column by column through a numpy view;
    every field of every entry must equal the field-by-field ctypes conversion."""
    from paper_1709_03013_gb300 import csg
    n = 37
    res = (csg._Result * n)()
    for k in range(n):
        r = res[k]
        r.d, r.status, r.N, r.R = 2 + 2 * (k % 2), -k if k % 5 == 0 else 0, 1000 + k, 3 * k
        for q in range(4):
            r.Nk[q] = k * 10 + q
        r.sum_m, r.W, r.combo, r.S = 2 ** 63 + k, 2 ** 40 + k, -7 * k, 0.5 * k - 3.25
    got = csg._results(res, n)
    want = [csg.Result.of(res[k]) for k in range(n)]
    assert got == want
    assert all(isinstance(x, csg.Result) and isinstance(x.Nk, tuple) for x in got)
    assert csg._results(res, 0) == []


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program that calls every declared entry point compiles with warnings as errors
    and links against the library (it is not run: no GPU here)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    names = _declared()
    body = "\n".join(f"    p[{k}] = (void (*)(void))&{n};" for k, n in enumerate(names))
    src = tmp_path / "use_csg.c"
    src.write_text(
        "#include <stdio.h>\n#include \"csg.h\"\n"
        f"int main(void) {{\n    void (*p[{len(names)}])(void);\n{body}\n"
        "    csg_result r;\n    (void)r;\n    printf(\"%p\\n\", (void *)p[0]);\n    return 0;\n}\n")
    libdir = os.path.dirname(lib._name)
    out = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-Wno-pedantic",
                          "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lcsg",
                          "-o", str(tmp_path / "use_csg")], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr


def test_no_fallback_without_library_or_device(lib, tmp_path):
    """The binding has no CPU path: a missing library is an ImportError that says how to build
    it, and without a usable GPU the context cannot be made (the failure is an error code, not
    a silent substitute)."""
    from paper_1709_03013_gb300 import csg
    saved, csg._lib = csg._lib, None   # as if nothing had been loaded yet
    try:
        with pytest.raises(ImportError, match="no CPU fallback"):
            csg.load(str(tmp_path / "libcsg.so"))
    finally:
        csg._lib = saved
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(csg.CsgError) as e:
        csg.Context(0)
    assert e.value.code in (csg.E_CUDA, csg.E_INVAL)


def _nvcc():
    import shutil
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


_MMA_KERNEL = r"""
#include <cstdint>
__global__ void k(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    if (threadIdx.x == 0)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n}\n"
                     :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
"""


@pytest.mark.parametrize("kind,arch,ok", [("i8", "103a", False), ("i8", "100a", True),
                                          ("f8f6f4", "103a", True), ("f16", "103a", True)])
def test_which_tensor_mma_kinds_exist_on_sm103a(tmp_path, kind, arch, ok):
    """Why the tensor form uses 0/1 operands in fp8/fp4 rather than int8: ptxas has no
    tcgen05 int8 MMA (kind::i8) for sm_103a, although it assembles one for sm_100a."""
    import subprocess
    src = tmp_path / "mma.cu"
    src.write_text(_MMA_KERNEL.replace("KIND", kind))
    r = subprocess.run([_nvcc(), "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", str(src),
                        "-o", str(tmp_path / "mma.o")], capture_output=True, text=True)
    assert (r.returncode == 0) == ok, r.stderr
    if not ok:
        assert "kind::i8" in r.stderr and "not supported" in r.stderr


def test_normal_build_compiles_no_bounds_checks(lib):
    words = (ctypes.c_uint64 * 8)()
    lib.csg_check_words.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.csg_check_words(ctypes.cast(words, ctypes.c_void_p), 8) == 0
