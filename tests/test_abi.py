"""CPU checks of the C ABI: the library builds, loads and exports every
function include/pint.h declares; argument validation needs no GPU."""
import ctypes
import os

import numpy as np

import pytest

from paper_2405_18964_gb300 import binding


def test_header_declares_the_boundary():
    names = binding.header_functions()
    for required in ["pint_create", "pint_set_data", "pint_apply_preconditioner", "pint_solve", "pint_destroy",
                     "pint_kkt_matvec", "pint_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libpint.so not built (run __graft_entry__.build())")
    L = binding.lib()
    missing = [n for n in binding.header_functions() if not hasattr(L, n)]
    assert missing == []
    # every declared function has a ctypes signature in the binding
    assert set(binding.header_functions()) == set(binding._SIGS)


def test_struct_layouts_match_header_field_order():
    src = open(binding.HEADER).read()
    body = src[src.index("typedef struct {\n  int kind;"):src.index("} pint_params;")]
    order = []
    for line in body.splitlines():
        line = line.split("/*")[0].strip().rstrip(";")
        if not line or line.startswith("typedef"):
            continue
        typ, names = line.split(None, 1)
        order += [n.strip() for n in names.split(",")]
    assert order == [f[0] for f in binding.Params._fields_]


def _header_struct_fields(src, name):
    """(field name, array length or 1) of `typedef struct { ... } name;` in
    the header, comments removed."""
    import re
    end = src.index("} " + name + ";")
    start = src.rindex("typedef struct {", 0, end)
    body = re.sub(r"/\*.*?\*/", "", src[start + len("typedef struct {"):end], flags=re.S)
    consts = {"PINT_PROF_CLASSES": binding.PROF_CLASSES and len(binding.PROF_CLASSES)}
    out = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        names = decl.split(None, 1)[1] if not decl.startswith(("long long", "unsigned")) else decl.split(None, 2)[2]
        for n in names.split(","):
            n = n.strip()
            if "[" in n:
                base, dim = n[:-1].split("[")
                out.append((base.strip(), consts.get(dim.strip(), None) or int(dim)))
            else:
                out.append((n, 1))
    return out


@pytest.mark.parametrize("cname,pyname", [("pint_solve_info", "SolveInfo"), ("pint_sizes", "Sizes"),
                                          ("pint_profile", "Profile"), ("pint_group_stats", "GroupStats"),
                                          ("pint_server_params", "ServerParams"),
                                          ("pint_server_stats", "ServerStats")])
def test_other_structs_match_header(cname, pyname):
    """Field order, array lengths and names of the result structures agree
    between include/pint.h and the ctypes binding."""
    fields = _header_struct_fields(open(binding.HEADER).read(), cname)
    py = getattr(binding, pyname)._fields_
    assert [f[0] for f in fields] == [f[0] for f in py]
    for (name, n), (_, ctype) in zip(fields, py):
        assert (getattr(ctype, "_length_", 1)) == n, name


def test_default_params_and_argument_validation():
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libpint.so not built")
    p = binding.default_params()
    assert (p.mg_cycles, p.cheb_steps, p.uzawa_steps, p.uzawa_mu, p.inner_tol) == (4, 10, 6, 0.75, 1e-2)
    h = ctypes.c_void_p()
    bad = binding.default_params(level=0)
    assert binding.lib().pint_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert b"level" in binding.lib().pint_last_error(None)
    for wind in (1, 2):
        bad = binding.default_params(kind=1, wind=wind, x0=0.0, x1=1.0)
        assert binding.lib().pint_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
        assert b"[-1,1]" in binding.lib().pint_last_error(None)
    bad = binding.default_params(kind=1, wind=4, x0=-1.0, x1=1.0)
    assert binding.lib().pint_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert b"wind" in binding.lib().pint_last_error(None)
    # a nodal wind goes through pint_create_wind, with finite values, on any domain
    nodal = binding.default_params(kind=1, wind=3, level=2, x0=0.0, x1=1.0)
    assert binding.lib().pint_create(ctypes.byref(nodal), None, ctypes.byref(h)) == 1
    assert b"pint_create_wind" in binding.lib().pint_last_error(None)
    w = np.zeros(2 * 81)
    wp = w.ctypes.data_as(ctypes.c_void_p)
    assert binding.lib().pint_create_wind(ctypes.byref(bad), wp, None, ctypes.byref(h)) == 1
    assert binding.lib().pint_create_wind(ctypes.byref(nodal), None, None, ctypes.byref(h)) == 1
    w[5] = np.nan
    assert binding.lib().pint_create_wind(ctypes.byref(nodal), wp, None, ctypes.byref(h)) == 5
    recirc = binding.default_params(kind=1, wind=1, level=2, x0=-1.0, x1=1.0)
    w[5] = 0.0
    assert binding.lib().pint_create_wind(ctypes.byref(recirc), wp, None, ctypes.byref(h)) == 1
    assert b"PINT_WIND_NODAL" in binding.lib().pint_last_error(None)
    bad = binding.default_params(prec=0, dft_mode=2)          # tensor-core DFT needs FP32
    assert binding.lib().pint_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert b"dft" in binding.lib().pint_last_error(None).lower()
    bad = binding.default_params(prec=1, dft_mode=3, n_t=300)  # and n_t <= 256
    assert binding.lib().pint_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    bad = binding.default_params(dft_mode=7)
    assert binding.lib().pint_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert binding.lib().pint_destroy(None) == 0


def test_device_estimate_counts_the_convection_tables():
    """pint_estimate_device_bytes (host only): Oseen with a wind needs the
    per-level convection stencils, the non-polynomial winds also their FP64
    node-order copies; invalid parameters give 0."""
    est = lambda **kw: binding.estimate_device_bytes(binding.default_params(**kw))
    base = dict(kind=1, level=6, n_t=64, x0=-1.0, x1=1.0, prec=1)
    none, recirc, two, nodal = (est(wind=w, **base) for w in (0, 1, 2, 3))
    assert 0 < none < recirc < two == nodal
    n2 = 2 * 64 + 1
    assert two - recirc >= n2 * n2 * 25 * 8          # at least the finest FP64 stencil table
    assert est(level=0) == 0


def _band_to_dense(st, n, hw):
    bw = 2 * hw + 1
    D = np.zeros((n * n, n * n))
    for i in range(n * n):
        ix, iy = i % n, i // n
        for k in range(bw * bw):
            jx, jy = ix + k % bw - hw, iy + k // bw - hw
            if 0 <= jx < n and 0 <= jy < n:
                D[i, jy * n + jx] = st[i, k]
    return D


@pytest.mark.parametrize("wind", [2, 3])
def test_host_convection_stencils_match_the_oracle(wind):
    """The FP64 convection stencils the library integrates on the host (two-
    vortex wind; a random nodal wind, injected to the coarse level) equal the
    oracle's skew-symmetric convection matrices on every level, Q2 and Q1."""
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("libpint.so not built (run __graft_entry__.build())")
    from oracle import fem
    level = 3
    N = 2 ** level
    W = np.random.default_rng(4).standard_normal((2, (2 * N + 1) ** 2)) if wind == 3 else None
    p = binding.default_params(kind=1, level=level, wind=wind, x0=-1.0, x1=1.0)
    name = ("nodal", W) if wind == 3 else "two_vortex"
    for l in range(level):
        n = N >> l
        q2, q1 = binding.convection_stencils(p, l, W)
        wf, skew = fem.wind_by_name(name, n, -1.0, 1.0)
        o = fem.assemble(n, -1.0, 1.0, wf, skew=skew)
        for st, A, m, hw in ((q2, o.N, 2 * n + 1, 2), (q1, o.Np, n + 1, 1)):
            ref = A.toarray()
            assert np.abs(_band_to_dense(st, m, hw) - ref).max() <= 1e-14 * np.abs(ref).max()
    with pytest.raises(binding.PintError):
        binding.convection_stencils(binding.default_params(kind=1, level=level, wind=1, x0=-1.0, x1=1.0))


class _FakeCudaTensor:
    """Stands in for a CUDA tensor in the binding's argument checks (no GPU)."""

    def __init__(self, numel):
        self._n = numel
        self.is_cuda = True
        self.dtype = "torch.complex128"

    def data_ptr(self):
        return 0

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n


class _FakeProblem:
    def __init__(self):
        self.h = None
        self.sizes = binding.Sizes(N=8, n_t=4, J=3, n_s=17 * 17, n_q=9 * 9, n_blk=4 * 289 + 2 * 81)


@pytest.mark.parametrize("method", ["mg_apply_noalloc", "component_apply"])
@pytest.mark.parametrize("which,good", [("mg_W", 289), ("mg_Kp", 81)])
def test_component_field_length_checked_before_any_call(method, which, good):
    """A field of the wrong length is refused on the host (ValueError) before
    the library is called: the C entry points take no length and would read
    or write past the end of the caller's buffer."""
    fn = getattr(binding.Problem, method)
    for n in (good - 1, good + 1, 0):
        with pytest.raises(ValueError):
            fn(_FakeProblem(), which, 0, _FakeCudaTensor(n), _FakeCudaTensor(good))
        with pytest.raises(ValueError):
            fn(_FakeProblem(), which, 0, _FakeCudaTensor(good), _FakeCudaTensor(n))
    assert binding.component_len(_FakeProblem().sizes, 6) == 4 * 289 + 2 * 81
