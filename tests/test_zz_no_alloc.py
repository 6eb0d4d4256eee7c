"""The allocation-free root reduction, vc_root_reduce_static, checked against
the regular entry point.

Some callers cannot call cudaMalloc: a process whose device memory belongs
to another allocator, or a latency-critical loop that must not risk the
device-wide synchronisation cudaMalloc / cudaFree can cause.  For them the
library keeps a fixed 2 MiB scratch array in device memory and this entry
point works only in it and in the caller's own buffers.

Each case calls the static entry point twice in a row through the C ABI and
requires both calls to agree with each other and with vc_solve_min's
root-phase statistics (forced vertices, induced subgraph size, greedy
bound); on small graphs the forced set plus the induced subgraph's optimum
must equal the oracle's optimum.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_18334_gb300 import build
    build.build()
    import paper_2512_18334_gb300 as vc
    return torch, vc


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def call_static(torch, vc, g, k=-1):
    dev = torch.device("cuda", torch.cuda.current_device())
    n, m2 = g.n, int(g.row_ptr[-1])
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).to(dev)
    col = torch.from_numpy(g.col if g.col.size else np.zeros(1, np.int32)).to(dev)
    forced = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    irp = torch.full((n + 1,), -1, dtype=torch.int32, device=dev)
    icol = torch.full((max(m2, 1),), -1, dtype=torch.int32, device=dev)
    iorig = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    info = torch.full((8,), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = vc._L.lib().vc_root_reduce_static(n, m2, _p(rp), _p(col), k, _p(forced), _p(irp), _p(icol),
                                            _p(iorig), _p(info), ctypes.c_void_p(stream.cuda_stream))
    assert rc == vc.VC_OK
    stream.synchronize()
    inf = info.cpu().numpy()
    assert inf[0] == vc.VC_OK
    nf, npr, m2p = int(inf[1]), int(inf[2]), int(inf[3])
    return (inf, set(forced.cpu().numpy()[:nf].tolist()), irp.cpu().numpy()[:npr + 1].copy(),
            icol.cpu().numpy()[:m2p].copy(), iorig.cpu().numpy()[:npr].copy())


CASES = [
    ("gnm_80_200_s0", lambda: gg.gnm(80, 200, 0)),
    ("gnm_80_200_s1", lambda: gg.gnm(80, 200, 1)),
    ("hub_components", lambda: gg.component_heavy(1, copies=8, copy_n=24, p=0.2, chain=3)),
    ("forest", lambda: gg.random_forest(3000, 4, 2)),
    ("chung_lu_50k", lambda: gg.chung_lu(50_000, 2.5, 6.0, 2000.0, 1000)),
    ("many_cores_12k", lambda: gg.disjoint_union([gg.gnm(40, 90, s) for s in range(300)])),
]


@pytest.mark.parametrize("name,make", CASES)
def test_static_matches_regular_entry_point(env, name, make):
    torch, vc = env
    g = make()
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    size, _, st = vc.solve_min(dg)
    dg.close()
    first = call_static(torch, vc, g)
    second = call_static(torch, vc, g)
    # two calls in a row agree exactly (the array keeps the last contents)
    assert np.array_equal(first[0], second[0])
    assert first[1] == second[1]
    for a, b in zip(first[2:], second[2:]):
        assert np.array_equal(a, b)
    inf, forced, irp, icol, iorig = first
    # the same root phase as vc_solve_min
    assert inf[1] == st["forced"] and len(forced) == st["forced"]
    assert inf[2] == st["n_induced"]
    assert inf[3] == 2 * st["m_induced"]
    assert inf[4] == st["greedy_size"]
    if inf[5]:
        assert inf[6] == size
    # the induced subgraph is G minus the forced vertices, isolated ones dropped
    keep = np.zeros(g.n, bool)
    deg_left = np.zeros(g.n, np.int64)
    fmask = np.zeros(g.n, bool)
    fmask[list(forced)] = True
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    live_e = ~fmask[src] & ~fmask[g.col]
    np.add.at(deg_left, src[live_e], 1)
    keep = deg_left > 0
    if not inf[5]:
        assert np.array_equal(iorig, np.nonzero(keep)[0])
        assert np.array_equal(np.diff(irp), deg_left[keep])
    if g.n <= 5000 and not inf[5]:
        sub_opt = oracle.mvc(int(inf[2]), irp, icol, node_budget=5_000_000)[0]
        assert inf[1] + sub_opt == size


def test_static_rejects_oversized_graph(env):
    torch, vc = env
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = vc._L.lib().vc_root_reduce_static(65537, 0, None, None, -1, None, None, None, None, _p(info), None)
    assert rc == vc.VC_ECAPACITY
    assert "capacity" in vc._L.strerror(rc)


@pytest.mark.parametrize("name,make", CASES[:4] + CASES[5:])
def test_static_decision_queries_match_regular_entry_point(env, name, make):
    # k = OPT and k = OPT - 1: the root phase bounded by k + 1, against the
    # regular decision call's root phase and answer
    torch, vc = env
    g = make()
    dg = vc.Graph.from_csr(g.row_ptr, g.col)
    opt, _, _ = vc.solve_min(dg)
    for k in (opt, opt - 1):
        if k < 0:
            continue
        yes, _, st = vc.solve_k(dg, k)
        inf, forced, _, _, _ = call_static(torch, vc, g, k=k)
        assert inf[1] == st["forced"] and len(forced) == st["forced"]
        assert inf[2] == st["n_induced"]
        if inf[5]:
            assert (inf[6] >= 0) == bool(yes)
            if yes:
                assert inf[6] <= k
    dg.close()


def test_static_reports_malformed_graphs(env):
    torch, vc = env
    # 0-1 and 1-2 listed once each: not mirrored
    rp = np.array([0, 1, 2, 2], np.int32)
    col = np.array([1, 2], np.int32)
    dev = torch.device("cuda", torch.cuda.current_device())
    trp = torch.from_numpy(rp).to(dev)
    tcol = torch.from_numpy(col).to(dev)
    bufs = [torch.full((8,), -1, dtype=torch.int32, device=dev) for _ in range(4)]
    info = torch.full((8,), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = vc._L.lib().vc_root_reduce_static(3, 2, _p(trp), _p(tcol), -1, _p(bufs[0]), _p(bufs[1]), _p(bufs[2]),
                                            _p(bufs[3]), _p(info), ctypes.c_void_p(stream.cuda_stream))
    assert rc == vc.VC_OK
    stream.synchronize()
    assert int(info[0]) == vc.VC_EINVAL


def test_static_call_allocates_nothing(env):
    # after a warm-up call on this device, the free device memory is the same
    # before and after two more calls (every buffer is the caller's, made first)
    torch, vc = env
    g = gg.chung_lu(20_000, 2.5, 6.0, 800.0, 3)
    dev = torch.device("cuda", torch.cuda.current_device())
    n, m2 = g.n, int(g.row_ptr[-1])
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    forced, irp, icol, iorig = (torch.empty((x,), dtype=torch.int32, device=dev) for x in (n, n + 1, m2, n))
    info = torch.empty((8,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    L = vc._L.lib()

    def call():
        return L.vc_root_reduce_static(n, m2, _p(rp), _p(col), -1, _p(forced), _p(irp), _p(icol), _p(iorig),
                                       _p(info), ctypes.c_void_p(stream.cuda_stream))

    assert call() == vc.VC_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert call() == vc.VC_OK and call() == vc.VC_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(info[0]) == vc.VC_OK
