"""The C-ABI library builds, loads and exports every symbol include/cyclicot.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cyclicot.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ot_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_13147_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ot_fold_cost", "ot_sinkhorn_reduced", "ot_sinkhorn_full", "ot_unfold_plan", "ot_value_and_grad",
              "ot_workspace_bytes", "ot_status_string", "ot_version", "ot_batch_prepare", "ot_batch_fold",
              "ot_batch_solve", "ot_batch_workspace_bytes", "ot_srot_reduced", "ot_srot_workspace_bytes",
              "ot_lot_reduced", "ot_lot_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_host_only_entry_points(libpath):
    from paper_2311_13147_gb300 import cyclicot as cy
    assert "sm_103a" in cy.version()
    assert cy.status_string(cy.OT_ERR_TIMEOUT).startswith("OT_ERR_TIMEOUT")
    assert cy.status_string(12345) == "unknown status"
    assert ctypes.sizeof(cy.ot_result) == 64
    assert ctypes.sizeof(cy.ot_problem_desc) == 48
    assert cy.ot_batch_workspace_bytes(0, 8) == 0
    assert cy.ot_batch_workspace_bytes(4, 100) > 0
    # the reduced LOT's workspace: FP64 row and column sums per problem (256-byte rounded); sizes above
    # the shared-memory tree's limit (m = 5120) are refused
    L = cy._lot_lib()
    assert L.ot_lot_workspace_bytes(3, 100) == (3 * 2 * 100 * 8 + 255) // 256 * 256
    assert L.ot_lot_workspace_bytes(1, 5120) > 0
    assert L.ot_lot_workspace_bytes(1, 5121) == 0 and L.ot_lot_workspace_bytes(0, 10) == 0
    assert cy._srot_lib().ot_srot_workspace_bytes(1024, 9) == 0   # N m above 8192


def test_binding_refuses_cpu_tensors(libpath):
    import torch
    from paper_2311_13147_gb300 import cyclicot as cy
    C = torch.zeros((2, 4, 4))
    with pytest.raises(ValueError):
        cy.ot_fold_cost(cy.OT_MIN, 4, 2, C_base=C, G=torch.zeros((4, 4)), kstar=torch.zeros((4, 4), dtype=torch.uint8))
    with pytest.raises(ValueError):
        cy.ot_lot_reduced(4, 2, torch.ones(4), torch.ones(4), torch.zeros((4, 4)))


def test_struct_layouts_match_header():
    """ot_options / ot_result field order in the binding follows the header."""
    from paper_2311_13147_gb300 import cyclicot as cy
    text = open(HEADER).read()
    for struct, cls in (("ot_options", cy.ot_options), ("ot_result", cy.ot_result),
                        ("ot_problem_desc", cy.ot_problem_desc)):
        body = re.search(r"typedef struct \{([^{}]*)\} " + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"\b([A-Za-z_0-9]+)\s*(?:\[\d+\])?\s*[;,]", body)
        assert [f[0] for f in cls._fields_] == fields


def test_batch_prepare_validates_the_table_on_the_host(libpath):
    """ot_batch_prepare checks every descriptor and the workspace before any device call, so the
    refusals below need no GPU (the workspace address is never dereferenced)."""
    from paper_2311_13147_gb300 import cyclicot as cy
    L = cy._batch_lib()
    D = cy.ot_problem_desc
    fake = ctypes.c_void_p(1 << 20)          # 256-byte aligned, never touched

    def prep(descs, ws=fake, nbytes=None):
        arr = (D * len(descs))(*descs)
        total_m = max(d.v_off + d.m for d in descs)
        n = cy.ot_batch_workspace_bytes(len(descs), total_m) if nbytes is None else nbytes
        return L.ot_batch_prepare(arr, len(descs), ws, n, None)

    good = [D(100, 4, 0.1, 100, 0, 0, 0, 100), D(37, 3, 0.05, 40, 10000, 100, 200, 237)]
    assert prep(good, ws=None) == cy.OT_ERR_ARG
    assert prep([D(100, 4, 0.1, 102, 0, 0, 0, 100)]) == cy.OT_ERR_ARG        # row stride not a multiple of 4
    assert prep([D(100, 4, 0.1, 96, 0, 0, 0, 100)]) == cy.OT_ERR_ARG         # stride shorter than the row
    assert prep([D(8193, 2, 0.1, 8196, 0, 0, 0, 8193)]) == cy.OT_ERR_ARG     # block wider than 8192
    assert prep([D(100, 4, 0.0, 100, 0, 0, 0, 100)]) == cy.OT_ERR_ARG        # eps <= 0
    assert prep([D(100, 257, 0.1, 100, 0, 0, 0, 100)]) == cy.OT_ERR_ARG      # N above 256
    assert prep([D(100, 4, 0.1, 100, 2, 0, 0, 100)]) == cy.OT_ERR_ARG        # cost offset not 16-byte aligned
    assert prep([D(0, 4, 0.1, 4, 0, 0, 0, 0)]) == cy.OT_ERR_ARG              # empty block
    need = cy.ot_batch_workspace_bytes(2, 137)
    assert prep(good, nbytes=need - 1) == cy.OT_ERR_WORKSPACE
    assert prep(good, ws=ctypes.c_void_p((1 << 20) + 16)) == cy.OT_ERR_WORKSPACE   # not 256-byte aligned
    arr = (D * 1)(good[0])
    assert L.ot_batch_prepare(arr, 0, fake, need, None) == cy.OT_ERR_ARG
    assert L.ot_batch_prepare(arr, 1025, fake, need, None) == cy.OT_ERR_ARG


def test_solver_and_fold_arguments_are_checked_on_the_host(libpath):
    """The fold and the reduced and full solvers refuse bad arguments before any device call, so
    each refusal below returns at once without touching the (fake) pointers."""
    from paper_2311_13147_gb300 import cyclicot as cy
    L = cy.lib()
    P = ctypes.c_void_p(1 << 20)            # 256-byte aligned, never dereferenced
    odd = ctypes.c_void_p((1 << 20) + 4)   # not 16-byte aligned
    NULL = None

    def opts(**kw):
        o = cy.options(0.1)
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def red(m=8, N=2, a=P, b=P, G=P, opt="ok", w=P, z=P, out=P):
        o = ctypes.byref(opts()) if opt == "ok" else opt
        return L.ot_sinkhorn_reduced(m, N, a, b, G, o, w, z, out, P, 1 << 20, NULL)

    for bad in (dict(m=0), dict(N=0), dict(a=NULL), dict(b=NULL), dict(G=NULL), dict(w=NULL), dict(z=NULL),
                dict(out=NULL), dict(opt=NULL), dict(G=odd)):
        assert red(**bad) == cy.OT_ERR_ARG, bad
    for field, value in (("eps", 0.0), ("max_iter", 0), ("check_every", 0), ("tol_l1", -1e-9), ("stop_norm", 7),
                         ("precision", 3), ("tile_override", 1)):
        assert red(opt=ctypes.byref(opts(**{field: value}))) == cy.OT_ERR_ARG, field

    def full(n=16, a=P, b=P, C=P, X=NULL, Y=NULL, f=P, g=P, out=P):
        return L.ot_sinkhorn_full(n, a, b, C, X, Y, ctypes.byref(opts()), f, g, out, P, 1 << 20, NULL)

    for bad in (dict(n=0), dict(a=NULL), dict(b=NULL), dict(f=NULL), dict(g=NULL), dict(out=NULL),
                dict(C=NULL), dict(C=NULL, X=P), dict(C=odd)):
        assert full(**bad) == cy.OT_ERR_ARG, bad

    def fold(mode=cy.OT_SOFTMIN, m=8, N=2, C=P, x=NULL, y=NULL, eps=0.1, G=P):
        return L.ot_fold_cost(mode, m, N, C, x, y, eps, G, NULL, NULL)

    for bad in (dict(m=0), dict(N=0), dict(G=NULL), dict(mode=9), dict(eps=0.0), dict(C=NULL), dict(C=NULL, x=P)):
        assert fold(**bad) == cy.OT_ERR_ARG, bad
    assert fold(mode=cy.OT_MIN, N=256) == cy.OT_ERR_UNSUPPORTED   # k* is one byte


def test_lot_srot_and_unfold_arguments_are_checked_on_the_host(libpath):
    """The reduced LOT and C-SROT solvers and the unfold refuse bad arguments (and, for the two
    solvers, short or misaligned workspaces and sizes above their limits) before any device call."""
    from paper_2311_13147_gb300 import cyclicot as cy
    P = ctypes.c_void_p(1 << 20)            # 256-byte aligned, never dereferenced
    NULL = None
    ok = ctypes.byref(cy.options(0.1))

    Lt = cy._lot_lib()
    need = Lt.ot_lot_workspace_bytes(2, 16)

    def lot(count=2, m=16, N=3, a=P, b=P, G=P, opt=ok, S=P, u=P, v=P, out=P, ws=P, nbytes=need):
        return Lt.ot_lot_reduced(count, m, N, a, b, G, opt, S, u, v, out, ws, nbytes, NULL)

    for bad in (dict(count=0), dict(m=0), dict(N=0), dict(a=NULL), dict(b=NULL), dict(G=NULL), dict(opt=NULL),
                dict(S=NULL), dict(u=NULL), dict(v=NULL), dict(out=NULL),
                dict(opt=ctypes.byref(cy.options(0.1, max_iter=0)))):
        assert lot(**bad) == cy.OT_ERR_ARG, bad
    assert lot(m=5121) == cy.OT_ERR_UNSUPPORTED
    for bad in (dict(ws=NULL), dict(nbytes=need - 1), dict(ws=ctypes.c_void_p((1 << 20) + 64))):
        assert lot(**bad) == cy.OT_ERR_WORKSPACE, bad

    Ls = cy._srot_lib()
    need = Ls.ot_srot_workspace_bytes(16, 2)

    def srot(m=16, N=2, a=P, b=P, C=P, opt=ok, w=P, z=P, out=P, ws=P, nbytes=need):
        return Ls.ot_srot_reduced(m, N, a, b, C, opt, w, z, out, ws, nbytes, NULL)

    for bad in (dict(m=0), dict(N=0), dict(a=NULL), dict(b=NULL), dict(C=NULL), dict(opt=NULL), dict(w=NULL),
                dict(z=NULL), dict(out=NULL), dict(opt=ctypes.byref(cy.options(0.0))),
                dict(opt=ctypes.byref(cy.options(0.1, max_iter=0))),
                dict(opt=ctypes.byref(cy.options(0.1, tol=-1.0)))):
        assert srot(**bad) == cy.OT_ERR_ARG, bad
    assert srot(m=1024, N=9) == cy.OT_ERR_UNSUPPORTED   # N m above 8192
    for bad in (dict(ws=NULL), dict(nbytes=need - 1), dict(ws=ctypes.c_void_p((1 << 20) + 64))):
        assert srot(**bad) == cy.OT_ERR_WORKSPACE, bad

    L = cy.lib()

    def unfold(mode=cy.OT_PLAN_EROT, m=8, N=2, S=P, z=P, C=P, x=NULL, y=NULL, k=P, eps=0.1, T=P):
        return L.ot_unfold_plan(mode, m, N, S, z, C, x, y, k, eps, 0, T, NULL)

    for bad in (dict(m=0), dict(N=0), dict(S=NULL), dict(T=NULL), dict(mode=7), dict(z=NULL), dict(eps=0.0),
                dict(C=NULL), dict(C=NULL, x=P), dict(mode=cy.OT_PLAN_LOT, k=NULL),
                dict(mode=cy.OT_PLAN_LOT, N=256)):
        assert unfold(**bad) == cy.OT_ERR_ARG, bad


def test_value_and_kernel_domain_arguments_are_checked_on_the_host(libpath):
    """ot_value_and_grad and the kernel-domain solver refuse bad arguments and workspaces before any
    device call (the unrolled adjoint only for its own missing inputs)."""
    from paper_2311_13147_gb300 import cyclicot as cy
    P = ctypes.c_void_p(1 << 20)            # 256-byte aligned, never dereferenced
    NULL = None
    L = cy.lib()
    big = 1 << 24

    def value(m=8, N=2, a=P, b=P, C=P, x=NULL, y=NULL, G=NULL, w=P, z=P, eps=0.1, adj=cy.OT_ADJ_ENVELOPE, T=0,
              out=P, dC=NULL, dx=NULL, dy=NULL, ws=P, nbytes=big):
        return L.ot_value_and_grad(m, N, a, b, C, x, y, G, w, z, eps, adj, T, out, NULL, NULL, dC, dx, dy, ws, nbytes,
                                   NULL)

    for bad in (dict(m=0), dict(N=0), dict(a=NULL), dict(b=NULL), dict(out=NULL), dict(eps=0.0), dict(C=NULL),
                dict(C=NULL, x=P), dict(dx=P), dict(C=NULL, x=P, y=P, dC=P), dict(adj=5), dict(w=NULL), dict(z=NULL),
                dict(adj=cy.OT_ADJ_UNROLLED, T=10), dict(adj=cy.OT_ADJ_UNROLLED, G=P, T=0)):
        assert value(**bad) == cy.OT_ERR_ARG, bad
    for bad in (dict(ws=NULL), dict(nbytes=64), dict(ws=ctypes.c_void_p((1 << 20) + 8))):
        assert value(**bad) == cy.OT_ERR_WORKSPACE, bad

    K = cy._kd_lib()
    need = K.ot_kdomain_workspace_bytes(256)

    def kd(m=256, G=P, ld=256, eps=0.1, nrhs=8, a=P, b=P, iters=4, z=P, ws=P, nbytes=need):
        return K.ot_kdomain_solve(m, G, ld, eps, nrhs, a, b, iters, z, NULL, ws, nbytes, NULL)

    for bad in (dict(m=0), dict(m=16385, ld=16385), dict(G=NULL), dict(ld=255), dict(eps=0.0), dict(nrhs=0),
                dict(nrhs=65), dict(a=NULL), dict(b=NULL), dict(iters=0), dict(z=NULL), dict(ws=NULL)):
        assert kd(**bad) == cy.OT_ERR_ARG, bad
    for bad in (dict(nbytes=need - 1), dict(ws=ctypes.c_void_p((1 << 20) + 128))):
        assert kd(**bad) == cy.OT_ERR_WORKSPACE, bad
