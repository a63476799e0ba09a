"""The legacy-VTK writer of pushed-forward micro fields (host code)."""
import numpy as np

from paper_2103_17040_gb300 import vtk


def _read_block(data, pos, n, dtype):
    nbytes = n * np.dtype(dtype).itemsize
    return np.frombuffer(data[pos:pos + nbytes], dtype=dtype), pos + nbytes


def test_quads_are_counterclockwise_and_cover_each_micro_mesh():
    Nm, nM = 3, 2
    conn = vtk.quad_connectivity(nM, Nm)
    assert conn.shape == (nM * Nm * Nm, 4)
    n1 = Nm + 1
    # coordinates of the reference nodes: every quad has positive orientation
    y1 = np.tile(np.arange(n1), n1) / Nm
    y2 = np.repeat(np.arange(n1), n1) / Nm
    for cell in conn:
        j = cell % (n1 * n1)
        x, y = y1[j], y2[j]
        area2 = np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)
        assert abs(area2 / 2 - 1.0 / Nm ** 2) < 1e-15
    # instance 1 uses only its own points
    assert conn[Nm * Nm:].min() == n1 * n1 and conn.max() == nM * n1 * n1 - 1


def test_file_round_trip(tmp_path):
    Nm, nM = 2, 3
    nm = (Nm + 1) ** 2
    rng = np.random.default_rng(0)
    xyv = rng.standard_normal((nM, nm, 3))
    path = tmp_path / "f.vtk"
    vtk.write_pushforward_vtk(str(path), xyv, Nm)
    data = path.read_bytes()
    assert data.startswith(b"# vtk DataFile Version 3.0\n")
    npts, ncell = nM * nm, nM * Nm * Nm
    i = data.index(b"POINTS %d float\n" % npts) + len(b"POINTS %d float\n" % npts)
    pts, i = _read_block(data, i, 3 * npts, ">f4")
    assert np.allclose(pts.reshape(-1, 3)[:, :2], xyv[:, :, :2].reshape(-1, 2).astype(np.float32))
    assert np.all(pts.reshape(-1, 3)[:, 2] == 0)
    hdr = b"\nCELLS %d %d\n" % (ncell, 5 * ncell)
    i = data.index(hdr, i) + len(hdr)
    cells, i = _read_block(data, i, 5 * ncell, ">i4")
    assert np.array_equal(cells.reshape(-1, 5)[:, 1:], vtk.quad_connectivity(nM, Nm))
    hdr = b"\nCELL_TYPES %d\n" % ncell
    i = data.index(hdr, i) + len(hdr)
    types, i = _read_block(data, i, ncell, ">i4")
    assert np.all(types == 9)
    hdr = b"LOOKUP_TABLE default\n"
    i = data.index(hdr, i) + len(hdr)
    vals, i = _read_block(data, i, npts, ">f4")
    assert np.allclose(vals, xyv[:, :, 2].ravel().astype(np.float32))
