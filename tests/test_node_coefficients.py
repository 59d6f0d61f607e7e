"""Host precompute of the per-node edge coefficients (fdtd_node_coefficients,
no GPU): every node's (ce_x, ce_y, ce_z) from the library's id volume and
table equals an independent numpy computation of the Model section's edge
permittivity (the mean of eps_r over the existing cells sharing the edge,
ce = 1/mean; 0 on PEC edges, on edges tangential to a PEC wall and on edges
that do not exist), bit for bit.  The library memoises nodes whose eight
cells and PEC bits repeat and merges per-plane tables; the cases cover
layered boards (long repeats), random materials (more than 256 triples, the
16-bit ids), PMC walls, PEC boxes and a per-cell PEC mask."""
import ctypes

import numpy as np
import pytest

from paper_1008_2602_gb300 import capi as C
from paper_1008_2602_gb300 import workloads as W

PEC, PMC = W.WALL_PEC, W.WALL_PMC


def library_coefficients(p, mask=None):
    g = C.fdtd_grid(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.courant, p.dt)
    b = C.fdtd_boundary()
    b.depth[:] = list(p.upml_depth)
    b.m, b.R0, b.kappa_max = p.upml_m, p.upml_R0, p.upml_kappa_max
    b.wall[:] = list(p.walls)
    mat = np.ascontiguousarray(p.mat, dtype=np.uint8)
    eps = np.ascontiguousarray(p.eps_r, dtype=np.float64)
    boxes = np.ascontiguousarray(p.pec_boxes, dtype=np.int32).reshape(-1, 6)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    ids = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1), np.uint16)
    table = np.zeros((65536, 4), np.float32)
    n = ctypes.c_int()
    C.fdtd_node_coefficients(ctypes.byref(g), mat.ctypes.data, eps.ctypes.data, len(eps),
                             boxes.ctypes.data if len(boxes) else None, len(boxes),
                             None if m is None else m.ctypes.data, ctypes.byref(b), ids.ctypes.data,
                             table.ctypes.data, len(table), ctypes.byref(n))
    return table[ids][..., :3], n.value


def reference_coefficients(p, mask=None):
    """Per node (k, j, i): ce of the x, y and z edges starting there, summed
    over the up-to-four cells in the same order as a scalar loop would."""
    nx, ny, nz = p.nx, p.ny, p.nz
    e = np.asarray(p.eps_r, np.float64)[p.mat]                      # [nz][ny][nx]
    ep = np.zeros((nz + 2, ny + 2, nx + 2))                          # cell (i, j, k) at [k+1][j+1][i+1]
    ep[1:-1, 1:-1, 1:-1] = e
    ok = np.zeros_like(ep)
    ok[1:-1, 1:-1, 1:-1] = 1.0
    K, J, I = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")

    def cell(i, j, k):          # eps and existence of cell (i, j, k); out-of-grid cells do not exist
        return ep[k + 1, j + 1, i + 1], ok[k + 1, j + 1, i + 1]

    def mean_inv(terms):
        s = np.zeros(K.shape)
        n = np.zeros(K.shape)
        for ii, jj, kk in terms:
            v, o = cell(np.clip(ii, -1, nx), np.clip(jj, -1, ny), np.clip(kk, -1, nz))
            s = s + v * o
            n = n + o
        with np.errstate(divide="ignore", invalid="ignore"):
            return (n / s).astype(np.float32)

    cx = mean_inv([(I, J - 1, K - 1), (I, J, K - 1), (I, J - 1, K), (I, J, K)])
    cy = mean_inv([(I - 1, J, K - 1), (I, J, K - 1), (I - 1, J, K), (I, J, K)])
    cz = mean_inv([(I - 1, J - 1, K), (I, J - 1, K), (I - 1, J, K), (I, J, K)])
    # edges that exist
    cx[I == nx] = 0
    cy[J == ny] = 0
    cz[K == nz] = 0
    # edges tangential to a PEC wall
    w = p.walls
    on_x = ((I == 0) & (w[0] == PEC)) | ((I == nx) & (w[1] == PEC))
    on_y = ((J == 0) & (w[2] == PEC)) | ((J == ny) & (w[3] == PEC))
    on_z = ((K == 0) & (w[4] == PEC)) | ((K == nz) & (w[5] == PEC))
    cx[on_y | on_z] = 0
    cy[on_x | on_z] = 0
    cz[on_x | on_y] = 0
    # PEC boxes (closed node boxes) and masked cells (1x1x1 boxes)
    boxes = [tuple(int(v) for v in bx) for bx in np.asarray(p.pec_boxes).reshape(-1, 6)]
    if mask is not None:
        boxes += [(i, i + 1, j, j + 1, k, k + 1) for k, j, i in zip(*np.nonzero(mask))]
    for i0, i1, j0, j1, k0, k1 in boxes:
        inside = (I >= i0) & (I <= i1) & (J >= j0) & (J <= j1) & (K >= k0) & (K <= k1)
        cx[inside & (I < i1)] = 0
        cy[inside & (J < j1)] = 0
        cz[inside & (K < k1)] = 0
    return np.stack([cx, cy, cz], axis=-1)


def _check(p, mask=None):
    got, n = library_coefficients(p, mask)
    ref = reference_coefficients(p, mask)
    assert got.shape == ref.shape
    bad = np.nonzero(np.any(got != ref, axis=-1))
    assert len(bad[0]) == 0, (len(bad[0]), [tuple(int(x) for x in t) for t in zip(*bad)][:5])
    return n


def test_layered_board_with_sheets():
    n = _check(W.small_pcb())
    assert n <= 256                     # 8-bit ids on the device


def test_multilayer_board_at_reduced_extent():
    _check(W.multilayer_board(scale=8, n_steps=10))


def test_random_materials_need_16_bit_ids():
    n = _check(W.random_problem(1, 37, 29, 23, upml=3, n_steps=10))
    assert n > 256


def test_pmc_walls_and_a_pec_mask():
    p = W.random_problem(5, 21, 17, 13, upml=0, n_steps=10).replace(
        upml_depth=(0,) * 6, walls=(PMC, PEC, PMC, PEC, PMC, PEC))
    mask = (np.random.default_rng(6).random((p.nz, p.ny, p.nx)) < 0.03).astype(np.uint8)
    _check(p, mask)


def test_errors():
    p = W.random_problem(1, 9, 8, 7, upml=2, n_steps=10)
    with pytest.raises(C.FdtdError):
        bad = p.replace(mat=np.full_like(p.mat, len(p.eps_r)))   # material id outside eps_r
        library_coefficients(bad)
    g = C.fdtd_grid(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.courant, p.dt)
    b = C.fdtd_boundary()
    b.depth[:] = list(p.upml_depth)
    b.m, b.R0, b.kappa_max = p.upml_m, p.upml_R0, p.upml_kappa_max
    b.wall[:] = list(p.walls)
    mat = np.ascontiguousarray(p.mat)
    eps = np.ascontiguousarray(p.eps_r, dtype=np.float64)
    ids = np.zeros((p.nz + 1, p.ny + 1, p.nx + 1), np.uint16)
    table = np.zeros((2, 4), np.float32)
    n = ctypes.c_int()
    with pytest.raises(C.FdtdError):   # far more than two distinct triples
        C.fdtd_node_coefficients(ctypes.byref(g), mat.ctypes.data, eps.ctypes.data, len(eps), None, 0, None,
                                 ctypes.byref(b), ids.ctypes.data, table.ctypes.data, 2, ctypes.byref(n))
