"""The allocation-free projection entry point, for callers that cannot allocate
device memory (a framework whose pool owns the whole GPU, or a loop that must not
pay for an allocation).  It must give the same projections as
pdcs_proj_cones_device, call after call, although its scratch array keeps the
previous call's contents."""
import numpy as np
import pytest

from paper_2505_00311_gb300 import build as B
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


def _cones(rng, n_blocks):
    types, dims = [], []
    for _ in range(n_blocks):
        t = int(rng.integers(0, 5))
        d = {0: int(rng.integers(1, 6)), 1: int(rng.integers(1, 6)), 2: int(rng.integers(1, 90)),
             3: int(rng.integers(2, 90)), 4: 3}[t]
        types.append(t)
        dims.append(d)
    return np.array(types, np.int32), np.array(dims, np.int64)


def _case(rng, n_blocks, scaled):
    types, dims = _cones(rng, n_blocks)
    m = int(dims.sum())
    v = rng.standard_normal(m) * np.exp(rng.normal(0, 1.5, m))
    d = None
    if scaled:
        d = np.exp(rng.normal(0, 1.0, m))
        o = 0
        for t, k in zip(types, dims):
            if t == P.CONE_RSOC:
                d[o + 1] = d[o]  # rotated SOC rows 1-2 share one scale
            o += k
    return v, d, types, dims


def test_noalloc_matches_the_allocating_entry_point():
    import torch
    B.build()
    rng = np.random.default_rng(31)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row per setting; the second uses a different (shorter) cone list, so
    # a stale offset or cone record left in the shared scratch would show up
    for dual in (0, 1):
        for scaled in (False, True):
            for n_blocks in (700, 90):
                v, d, types, dims = _case(rng, n_blocks, scaled)
                tv = torch.tensor(v, dtype=torch.float64, device="cuda")
                td = None if d is None else torch.tensor(d, dtype=torch.float64, device="cuda")
                ref = torch.empty_like(tv)
                got = torch.full_like(tv, float("nan"))
                dp = 0 if td is None else td.data_ptr()
                P.pdcs_proj_cones_device(tv.data_ptr(), dp, v.size, types, dims, dual, ref.data_ptr(), stream)
                st = P.pdcs_proj_cones_device_noalloc(tv.data_ptr(), dp, v.size, types, dims, dual, got.data_ptr(),
                                                      stream)
                assert st == P.OK
                torch.cuda.synchronize()
                r, g = ref.cpu().numpy(), got.cpu().numpy()
                o = 0
                for t, k in zip(types, dims):
                    blk = slice(o, o + k)
                    assert np.linalg.norm(g[blk] - r[blk]) <= 1e-12 * max(np.linalg.norm(v[blk]), 1e-300), (t, k)
                    o += k


def test_noalloc_large_soc_blocks_match():
    """SOC and RSOC blocks of dimension 130-600, where the allocating entry point switches to
    its mixed-precision path with scratch while this one stays on its FP64 search: primal and
    dual, unscaled and scaled, within the same 1e-12 of each other, two calls in a row."""
    import torch
    B.build()
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream().cuda_stream
    for dual in (0, 1):
        for scaled in (False, True):
            for n_blocks in (40, 25):
                types = rng.choice([P.CONE_SOC, P.CONE_RSOC], n_blocks).astype(np.int32)
                dims = rng.integers(130, 601, n_blocks).astype(np.int64)
                m = int(dims.sum())
                v = rng.standard_normal(m) * np.exp(rng.normal(0, 1.5, m))
                # put the first entry of each block where the projection is a genuine root search
                o = 0
                for k in dims:
                    v[o] = rng.uniform(-1.0, 1.0) * np.linalg.norm(v[o + 1:o + k])
                    o += k
                d = None
                if scaled:
                    d = np.exp(rng.normal(0, 1.0, m))
                    o = 0
                    for t, k in zip(types, dims):
                        if t == P.CONE_RSOC:
                            d[o + 1] = d[o]
                        o += k
                tv = torch.tensor(v, dtype=torch.float64, device="cuda")
                td = None if d is None else torch.tensor(d, dtype=torch.float64, device="cuda")
                ref = torch.empty_like(tv)
                got = torch.full_like(tv, float("nan"))
                dp = 0 if td is None else td.data_ptr()
                P.pdcs_proj_cones_device(tv.data_ptr(), dp, m, types, dims, dual, ref.data_ptr(), stream)
                st = P.pdcs_proj_cones_device_noalloc(tv.data_ptr(), dp, m, types, dims, dual, got.data_ptr(), stream)
                assert st == P.OK
                torch.cuda.synchronize()
                r, g = ref.cpu().numpy(), got.cpu().numpy()
                o = 0
                for t, k in zip(types, dims):
                    blk = slice(o, o + k)
                    assert np.linalg.norm(g[blk] - r[blk]) <= 1e-12 * np.linalg.norm(v[blk]), (t, k)
                    o += k


def test_noalloc_calls_allocate_nothing():
    """After a first call (which looks up the scratch array's address), 100 calls with
    different cone lists leave the device's free memory and torch's allocator unchanged."""
    import torch
    B.build()
    rng = np.random.default_rng(5)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [_case(rng, int(n), bool(n % 2)) for n in rng.integers(50, 400, 100)]
    bufs = []
    for v, d, types, dims in cases:
        tv = torch.tensor(v, dtype=torch.float64, device="cuda")
        td = None if d is None else torch.tensor(d, dtype=torch.float64, device="cuda")
        bufs.append((tv, td, torch.empty_like(tv), types, dims))
    tv, td, out, types, dims = bufs[0]
    assert P.pdcs_proj_cones_device_noalloc(tv.data_ptr(), 0 if td is None else td.data_ptr(), tv.numel(), types,
                                            dims, 0, out.data_ptr(), stream) == P.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for k, (tv, td, out, types, dims) in enumerate(bufs):
        st = P.pdcs_proj_cones_device_noalloc(tv.data_ptr(), 0 if td is None else td.data_ptr(), tv.numel(), types,
                                              dims, k % 2, out.data_ptr(), stream)
        assert st == P.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_oversized_and_malformed_lists():
    import torch
    B.build()
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    s = torch.cuda.current_stream().cuda_stream
    n = P.NOALLOC_MAX_CONES + 1
    st = P.pdcs_proj_cones_device_noalloc(v.data_ptr(), 0, n, np.ones(n, np.int32), np.ones(n, np.int64), 0,
                                          out.data_ptr(), s)
    assert st == P.ERR_INVALID
    st = P.pdcs_proj_cones_device_noalloc(v.data_ptr(), 0, 8, np.array([4], np.int32), np.array([8], np.int64), 0,
                                          out.data_ptr(), s)
    assert st == P.ERR_INVALID
