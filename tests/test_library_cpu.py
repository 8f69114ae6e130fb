"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function include/pne.h declares.  No GPU compute is issued."""
import os
import re

import numpy as np
import pytest

from paper_2512_10910_gb300 import build as B
from paper_2512_10910_gb300 import pne

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(pne_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = pne.load_library()
    declared = _declared()
    assert len(declared) >= 12
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    for n in _declared():
        assert hasattr(pne, n), n


def test_ctx_create_without_a_device_reports_an_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pne.PneError) as ei:
        pne.pne_ctx_create(0)
    assert ei.value.status == pne.PNE_ECUDA


def test_struct_layouts():
    import ctypes
    # pne_network: 2 ints, 4 pointers, data, data_off, 2 ints (LP64)
    assert ctypes.sizeof(pne.Network) == 8 + 4 * 8 + 8 + 8 + 8
    assert ctypes.sizeof(pne.PartitionOpts) == 56
    assert ctypes.sizeof(pne.EnumOpts) == 16
    # pne_trace_entry: name[32], kind, stream, t0_ms, t1_ms
    assert ctypes.sizeof(pne.TraceEntry) == 32 + 4 + 4 + 8 + 8


def test_tensor_offsets_match_per_site_leg_products():
    # the binding packs data_off from a segmented product over the CSR legs;
    # it must equal the per-site product of leg dimensions, including sites
    # without legs and open legs
    import numpy as np
    from paper_2512_10910_gb300 import inputs as I
    graphs = [I.square_lattice(6, 5, 3), I.cubic_lattice(3, 3, 3, 2), I.grid_graph(1, [], []),
              I.grid_graph(4, [(0, 1), (1, 2)], [2, 5]),          # site 3 has no legs
              I.grid_graph(5, [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 2), (0, 1), (3, 1)],
                           [2, 3, 2, 2, 3, 2, 2, 3]),
              I.with_open_legs(I.square_lattice(3, 3, 2), [(0, 3), (4, 2)])]
    for g in graphs:
        sizes, off = pne._offsets(g)
        want = [int(np.prod(g.leg_dims(v))) for v in range(g.n_sites)]
        assert list(sizes) == want
        assert off[0] == 0 and list(np.diff(off)) == want


def test_results_sequence_converts_on_access():
    arr = (pne.Result * 3)()
    for i in range(3):
        arr[i].log_abs = float(i)
        arr[i].n_orders = 2
        arr[i].c[0], arr[i].c[1] = 1.0, 0.5 * i
    res = pne.Results(arr)
    assert len(res) == 3
    assert res[-1]["log_abs"] == 2.0 and res[0]["log_abs"] == 0.0
    assert [r["log_abs"] for r in res] == [0.0, 1.0, 2.0]
    assert [r["log_abs"] for r in res[1:]] == [1.0, 2.0]
    assert list(res[2]["c"]) == [1.0, 1.0]
    assert res[1] is res[1]                       # built once
    (a, b, c) = res
    assert c["log_abs"] == 2.0
    with pytest.raises(IndexError):
        res[3]


def test_open_tensor_assembles_set_major_row_major_slices():
    import math
    import numpy as np
    dims, n_sets = (2, 3), 2
    arr = (pne.Result * (n_sets * 6))()
    want = np.zeros((n_sets,) + dims)
    for r in range(n_sets * 6):
        b, a = divmod(r, 6)
        i, j = divmod(a, 3)
        v = (-1.0) ** r * (1.0 + r)
        want[b, i, j] = v
        arr[r].sign = 1 if v > 0 else -1
        arr[r].log_abs = math.log(abs(v))
        arr[r].n_orders = 1
    arr[5].sign = 0                      # a zero result (Z_ref = 0 on that slice)
    want[0, 1, 2] = 0.0
    got = pne.open_tensor(pne.Results(arr), dims, n_sets)
    np.testing.assert_allclose(got, want, rtol=1e-15)


def test_noalloc_bp_rejects_an_oversized_network_on_the_host():
    # the scratch-size check runs on the host before any CUDA call: a network
    # whose messages alone exceed PNE_NOALLOC_SCRATCH_BYTES (8 MiB) comes back
    # with PNE_EINVAL; the device pointers are never dereferenced, so stand-ins
    # serve (no GPU is touched)
    import numpy as np
    from paper_2512_10910_gb300 import inputs as I
    g = I.square_lattice(4, 4, 2)
    B = 4096
    ns, keep = pne.network_struct(g, data=np.zeros(1), n_batch=B)
    ns.data = 0x1000
    ns.data_on_device = 1
    with pytest.raises(pne.PneError) as e:
        pne.pne_bp_messages_noalloc(ns, 0x2000, 1e-13, 10000)
    assert e.value.status == pne.PNE_EINVAL and "PNE_NOALLOC_SCRATCH_BYTES" in str(e.value)
    del keep


def test_open_tensor_assembly_keeps_huge_values_as_mantissa_and_scale():
    # slices whose |Z_K| is far beyond the FP64 range (ln|Z| ~ 800): the
    # library's assembly returns mantissas in [-1, 1] and the log scale
    import math
    import numpy as np
    n_sets, n_open = 2, 4
    arr = (pne.Result * (n_sets * n_open))()
    logs = [800.0, 801.5, 799.0, 802.25, -3.0, -2.0, float("-inf"), -1.0]
    signs = [1, -1, 1, 1, -1, 1, 1, 1]
    for r in range(n_sets * n_open):
        arr[r].sign = signs[r]
        arr[r].log_abs = logs[r]
        arr[r].n_orders = 1
    mant, ls = pne.pne_open_tensor_assemble(pne.Results(arr), n_sets, [n_open])
    assert ls[0] == 802.25 and ls[1] == -1.0
    np.testing.assert_allclose(mant[0], [math.exp(-2.25), -math.exp(-0.75), math.exp(-3.25), 1.0], rtol=1e-15)
    np.testing.assert_allclose(mant[1], [-math.exp(-2.0), math.exp(-1.0), 0.0, 1.0], rtol=1e-15)
    full = pne.open_tensor(pne.Results(arr), [n_open], n_sets)     # plain values: +-inf beyond range
    assert np.isinf(full[0]).all() and np.isfinite(full[1]).all()


def test_strip_struct_layouts_match_the_header(tmp_path):
    # the C compiler's sizes and offsets of the strip-expansion structs
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "lay.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pne.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pne_strip_opts), sizeof(pne_strip_result),\n'
                   ' offsetof(pne_strip_result, log_z), offsetof(pne_strip_result, sign_z),\n'
                   ' offsetof(pne_strip_result, messages), offsetof(pne_strip_result, eig_change),\n'
                   ' offsetof(pne_strip_result, iters), offsetof(pne_strip_opts, arithmetic));\nreturn 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    R, O = pne.StripResult, pne.StripOpts
    want = [ctypes.sizeof(O), ctypes.sizeof(R), R.log_z.offset, R.sign_z.offset, R.messages.offset,
            R.eig_change.offset, R.iters.offset, O.arithmetic.offset]
    assert got == want


def test_batch_and_partition_opts_layouts_match_the_header(tmp_path):
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "lay.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pne.h"\nint main(void){\n'
                   'printf("%zu %zu %d %d %zu %zu %zu %zu\\n", sizeof(pne_batch_opts),\n'
                   ' offsetof(pne_batch_opts, schedule), PNE_SCHED_HANDLE, PNE_SCHED_LARGEST_FIRST,\n'
                   ' sizeof(pne_partition_opts), offsetof(pne_partition_opts, use_user_projectors),\n'
                   ' offsetof(pne_partition_opts, user_u), offsetof(pne_partition_opts, user_v));\nreturn 0;}\n')
    exe = tmp_path / "lay"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    B, P = pne.BatchOpts, pne.PartitionOpts
    assert got == [ctypes.sizeof(B), B.schedule.offset, pne.PNE_SCHED_HANDLE, pne.PNE_SCHED_LARGEST_FIRST,
                   ctypes.sizeof(P), P.use_user_projectors.offset, P.user_u.offset, P.user_v.offset]


def test_user_projector_options_point_at_the_callers_vectors():
    # host-side marshalling only: flat FP64 arrays, equal lengths, flag set
    import ctypes
    u = np.arange(6, dtype=np.float64)
    v = np.arange(6, 12, dtype=np.float64)
    o, keep = pne.user_projector_opts(u, v, arithmetic=1)
    assert o.use_user_projectors == 1 and o.arithmetic == 1
    assert ctypes.addressof(o.user_u.contents) == keep[0].ctypes.data
    assert [o.user_v[i] for i in range(6)] == list(v)
    with pytest.raises(ValueError):
        pne.user_projector_opts(u, v[:5])
