"""The largest grids: more values than 32-bit offsets reach.

Past 2^31 stored values the tiled kernel still stores V_{n+1} through 32-bit
indices, counted in float4 units (they reach 2^34 values), and from 2^32
cells on the generic kernel splits cell indices with 64-bit divisions instead
of the 32-bit multiply-high ones.  Each case takes
V0 from its (x, y) field (Eq. init_V depends on the position only), given as
that field (the broadcast-V0 variants) or replicated in 4D on the device, runs
two steps with the kernel AUTO picks (the tiled one for FP32 and Q5.27, the
generic one for FP64) or the generic one, and checks each step against the
oracle's step at sampled cells: random cells, every face, edge and corner
class, and the cells on both sides of the 2^31 and 2^32 flat indices.

The oracle reads, for a cell, only the cell and its neighbours one point away
on each axis (wrapping in theta), and V0 at the cell.  So the host arrays it
is given are anonymous zero-filled mappings of the full size, written only at
those points, with huge pages declined: only the pages written are backed by
memory (a few hundred MB at most).  The device values are read back into a
device buffer and gathered there.

Device memory: the FP64 case holds 3 x 38.7 GB of grid buffers plus a 35 GB
read-back buffer (about 151 GB of the 288 GB); a 4D V0 input (FP32, 17.7 GB)
is freed before the read-back buffer is taken.
"""
import mmap

import numpy as np
import pytest

import oracle
from paper_2012_04011_gb300 import scenes

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CASES = [  # precision, grid, kernel ("auto" or "generic"), V0 given as its (x, y) field or in 4D
    ("fp32", (1536, 1536, 32, 33), "auto", "xy"),  # 2.49e9 cells, 2.7e9 stored values
    ("fp32", (1536, 1536, 32, 33), "generic", "xy"),  # 32-bit cell indices above 2^31
    ("fp32", (2048, 2048, 32, 33), "auto", "xy"),  # 4.43e9 cells, 4.8e9 stored values
    ("fp32", (2048, 2048, 32, 33), "auto", "4d"),
    ("fp32", (2048, 2048, 32, 33), "generic", "xy"),  # 64-bit cell indices
    ("q527", (2048, 2048, 32, 33), "auto", "xy"),
    ("q527", (2048, 2048, 32, 33), "auto", "4d"),
    ("q527", (2048, 2048, 32, 33), "generic", "xy"),
    ("fp64", (2048, 2048, 32, 33), "auto", "xy"),  # generic (the FP64 path)
    ("fp32", (8, 4096, 4096, 36), "auto", "4d"),  # x planes of 6e8 values
]


@pytest.fixture(scope="module")
def hj():
    from paper_2012_04011_gb300 import _build
    _build.build()
    from paper_2012_04011_gb300 import hj as mod
    return mod


def sample_cells(n, rng):
    N1, N2, N3, N4 = n
    ncell = N1 * N2 * N3 * N4
    cells = list(rng.integers(0, ncell, 3000))
    for i in (0, 1, N1 // 2, N1 - 2, N1 - 1):
        for j in (0, 1, N2 // 2, N2 - 2, N2 - 1):
            for k in (0, 1, N3 - 1):
                for l in (0, 1, N4 - 2, N4 - 1):
                    cells.append(((i * N2 + j) * N3 + k) * N4 + l)
    for edge in (1 << 31, 1 << 32, ncell):
        cells += [c for c in range(edge - 2, edge + 2) if 0 <= c < ncell]
    return np.unique(np.array(cells, dtype=np.int64))


def stars(n, cells):
    """The cells and their neighbours one point away on each axis (theta
    wraps; the other axes stop at the boundary)."""
    N1, N2, N3, N4 = n
    strides = (N2 * N3 * N4, N3 * N4, N4, 1)
    idx = np.stack(np.unravel_index(cells, n), axis=1)
    out = [cells]
    for d in range(4):
        for step in (-1, 1):
            j = idx[:, d] + step
            if d == 3:
                out.append(cells + ((j % N4) - idx[:, d]) * strides[d])
            else:
                ok = (j >= 0) & (j < n[d])
                out.append(cells[ok] + step * strides[d])
    return np.unique(np.concatenate(out))


def lazy_zeros(count, dtype):
    """A zero-filled array backed by an anonymous mapping: pages are backed by
    memory only once written, in base-page units (no huge pages)."""
    mm = mmap.mmap(-1, count * np.dtype(dtype).itemsize, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    if hasattr(mmap, "MADV_NOHUGEPAGE"):
        mm.madvise(mmap.MADV_NOHUGEPAGE)
    return np.frombuffer(mm, dtype=dtype)


def host_view(torch, dev, where, like):
    """A zero-filled host array of the full size holding the device values at
    `where` (only those pages are touched)."""
    h = lazy_zeros(dev.numel(), like)
    h[where] = dev[torch.from_numpy(where).to(dev.device)].cpu().numpy()
    return h


@pytest.mark.parametrize("prec,n,kernel,v0form", CASES)
def test_sampled_steps_on_grids_past_32_bit_offsets(hj, prec, n, kernel, v0form):
    torch = pytest.importorskip("torch")
    p = {"fp32": hj.HJ_FP32, "fp64": hj.HJ_FP64, "q527": hj.HJ_Q527}[prec]
    tdt = {"fp32": torch.float32, "fp64": torch.float64, "q527": torch.int32}[prec]
    ndt = {"fp32": np.float64, "fp64": np.float64, "q527": np.int32}[prec]
    ncell = int(np.prod(n))
    grid = scenes.GridSpec(n)
    scene = scenes.random_scene(np.random.default_rng(101), 12)
    v0_xy = scenes.signed_distance_xy(grid, scene)
    P = oracle.Problem(n, grid.lo, grid.hi, grid.periodic, oracle.DYN_CAR4D, (scenes.A_MAX, scenes.W_MAX))
    cells = sample_cells(n, np.random.default_rng(7))
    star = stars(n, cells)
    T, cfl = 1.0, scenes.CFL
    out = None
    try:
        with hj.Grid(n, grid.lo, grid.hi, grid.periodic, p) as g:
            g.set_dynamics(hj.HJ_DYN_CAR4D, (scenes.A_MAX, scenes.W_MAX))
            if v0form == "xy":
                src = v0_xy
                g.set_initial_value_xy(v0_xy)
            else:  # the field replicated over v and theta on the device, in FP32
                src = v0_xy.astype(np.float32).astype(np.float64)
                v4 = torch.from_numpy(v0_xy).to("cuda", torch.float32)[:, :, None, None].expand(*n).contiguous()
                hj.hj_set_initial_value_device(g.handle, v4)
                del v4
                torch.cuda.empty_cache()
            if kernel == "generic":
                g.set_kernel(hj.HJ_KERNEL_GENERIC)
            want_kernel = hj.HJ_KERNEL_TILED if kernel == "auto" and prec != "fp64" else hj.HJ_KERNEL_GENERIC
            assert g.info().kernel == want_kernel
            out = torch.empty(ncell, dtype=tdt, device="cuda")
            g.read_value_device(out)  # V0 as stored (n = 0)
            Vn = host_view(torch, out, star, ndt)
            v0_at = Vn[cells].copy()
            # V0 is the (x, y) field replicated over v and theta, in the grid's precision
            i, j = np.unravel_index(cells, n)[:2]
            want0 = {"fp32": lambda a: a.astype(np.float32), "fp64": lambda a: a, "q527": oracle.to_q527}[prec]
            assert np.array_equal(v0_at, want0(src[i, j]))
            V0h = lazy_zeros(ncell, ndt)  # the oracle reads V0 only at the sampled cells
            V0h[cells] = v0_at
            for _ in range(2):
                st = g.advance_brt(T, cfl, 1)
                assert st.steps == 1 and st.kernel == want_kernel
                g.read_value_device(out)
                got = out[torch.from_numpy(cells).to(out.device)].cpu().numpy()
                if prec == "q527":
                    want = oracle.step_cells_q527(P, Vn, V0h, st.dt_last, cells)
                    assert np.array_equal(got, want)
                else:
                    want = oracle.step_cells(P, Vn, V0h, st.dt_last, cells)
                    tol = 1e-12 if prec == "fp64" else 8 * np.finfo(np.float32).eps * float(np.abs(v0_xy).max())
                    assert float(np.abs(got.astype(np.float64) - want).max()) <= tol
                    assert np.all(got <= v0_at)
                del Vn
                Vn = host_view(torch, out, star, ndt)
    finally:
        del out
        torch.cuda.empty_cache()
