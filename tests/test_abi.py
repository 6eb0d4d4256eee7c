"""The C-ABI library builds for sm_103a, loads, and exports every function the
public header declares; the ctypes structs match the C layout.  No GPU
needed (no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vc_gb300.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_18334_gb300 import build
    build.build()
    import paper_2512_18334_gb300._lib as L
    return L


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["vc_load_csr", "vc_solve_min", "vc_solve_k", "vc_free", "vc_strerror",
                 "vc_solve_batch", "vc_load_csr_device", "vc_options_default"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vc_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    L = lib.lib()
    for f in declared_functions():
        assert hasattr(L, f)
        assert f in lib.SIGNATURES, f"binding lacks a signature for {f}"


def test_build_targets_sm_103a_only():
    from paper_2512_18334_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_without_gpu(lib):
    L = lib.lib()
    assert L.vc_strerror(0).decode() == "ok"
    assert "malformed" in L.vc_strerror(-1).decode()
    assert L.vc_strerror(-99).decode() == "unknown status"


def test_struct_layout_matches_header(lib, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "vc_gb300.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(vc_options), offsetof(vc_options, node_budget),
         sizeof(vc_stats), offsetof(vc_stats, n), offsetof(vc_stats, ms_root),
         offsetof(vc_stats, comp_hist));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    O, S = lib.Options, lib.Stats
    assert vals == [ctypes.sizeof(O), O.node_budget.offset, ctypes.sizeof(S), S.n.offset,
                    S.ms_root.offset, S.comp_hist.offset]


def test_options_default_without_gpu(lib):
    import paper_2512_18334_gb300 as vc
    o = vc.options()
    assert o.use_components == 1 and o.load_balance == 1 and o.idle_timeout_ms == 60000
    assert o.cuda_graph == 1   # the search phase is replayed from a CUDA graph by default
    assert o.capacity_retries == 2
    assert o.crown == 0 and o.disable_bounds == 0 and o.disable_root_rules == 0 and o.disable_dyn_bounds == 0


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2512_18334_gb300._lib as L
    monkeypatch.setattr(L, "_LIB_FILE", str(tmp_path / "nope.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(ImportError):
        L.lib()


def test_every_field_offset_matches_header(lib, tmp_path):
    # each ctypes mirror against gcc's layout of the C declaration, field by field
    structs = {"vc_options": lib.Options, "vc_stats": lib.Stats, "vc_server_config": lib.ServerConfig,
               "vc_server_result": lib.ServerResult, "vc_server_stats": lib.ServerStats}
    lines = []
    for cname, cls in structs.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
    src = tmp_path / "fields.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "vc_gb300.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "fields"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    want = []
    for cls in structs.values():
        want.append(ctypes.sizeof(cls))
        want.extend(getattr(cls, f).offset for f, _ in cls._fields_)
    assert vals == want


def test_server_config_default_without_gpu(lib):
    c = lib.ServerConfig()
    assert lib.lib().vc_server_config_default(ctypes.byref(c)) == 0
    assert c.max_inflight == 1024 and c.max_induced == 2048 and c.quantum_us == 2000
    assert c.dtype_bytes == 2 and c.use_components == 1 and c.arena_bytes == 2 << 30
    assert lib.lib().vc_server_config_default(None) == -1


def test_trim_without_gpu(lib):
    # nothing pooled yet in this process: frees nothing and needs no device
    assert lib.lib().vc_trim() == 0


def test_stats_dict_reads_every_field():
    # the binding converts vc_stats with one struct unpack built from the
    # ctypes layout; every field must come back as ctypes itself reads it
    import random
    from paper_2512_18334_gb300 import _lib as L
    rng = random.Random(3)
    for _ in range(20):
        st = L.Stats()
        for name, ct in L.Stats._fields_:
            if issubclass(ct, ctypes.Array):
                arr = getattr(st, name)
                for i in range(ct._length_):
                    arr[i] = rng.randrange(-2**40, 2**40) if ct._type_ is ctypes.c_int64 else rng.randrange(-2**31, 2**31)
            elif ct is ctypes.c_double:
                setattr(st, name, rng.uniform(-1e6, 1e6))
            elif ct is ctypes.c_int64:
                setattr(st, name, rng.randrange(-2**62, 2**62))
            else:
                setattr(st, name, rng.randrange(-2**31, 2**31))
        d = st.to_dict()
        for name, ct in L.Stats._fields_:
            if name == "comp_hist":
                assert d[name] == {i + 2: st.comp_hist[i] for i in range(16) if st.comp_hist[i]}
            elif name == "root_cycles":
                assert d[name] == list(st.root_cycles)
            elif name == "phase_cycles":
                assert d[name] == {L.PHASES[i]: st.phase_cycles[i] for i in range(6)}
            else:
                assert d[name] == getattr(st, name), name
