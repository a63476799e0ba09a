"""Legacy-VTK file of pushed-forward micro fields (host post-processing).

The paper renders its two-scale solutions with ParaView (Sec. 3.6).  Without a
graphics stack here, the library computes the push-forward on the GPU
(``TwoScale.pushforward``: every micro node at its physical, translated and
scaled position with its value) and this module writes that buffer as a VTK
unstructured grid of quadrilaterals that ParaView reads.
"""
from __future__ import annotations

import numpy as np

VTK_QUAD = 9


def quad_connectivity(nM: int, Nm: int) -> np.ndarray:
    """[nM * Nm * Nm, 4] point indices of the micro cells, counter-clockwise,
    micro node (p, q) of instance i at point i (Nm+1)^2 + p + (Nm+1) q."""
    n1 = Nm + 1
    a, b = np.meshgrid(np.arange(Nm), np.arange(Nm), indexing="xy")
    j0 = (a + n1 * b).ravel()
    cell = np.stack([j0, j0 + 1, j0 + 1 + n1, j0 + n1], axis=1)
    base = (np.arange(nM) * n1 * n1)[:, None, None]
    return (cell[None, :, :] + base).reshape(-1, 4)


def write_pushforward_vtk(path: str, xyv: np.ndarray, Nm: int, title: str = "two-scale micro fields") -> None:
    """xyv: [nM, (Nm+1)^2, 3] = (X1, X2, v) as returned by TwoScale.pushforward."""
    xyv = np.asarray(xyv, dtype=np.float64)
    nM, nm, three = xyv.shape
    if three != 3 or nm != (Nm + 1) ** 2:
        raise ValueError("xyv must be [nM, (Nm+1)^2, 3]")
    npts = nM * nm
    pts = np.zeros((npts, 3), dtype=">f4")
    pts[:, 0] = xyv[:, :, 0].ravel()
    pts[:, 1] = xyv[:, :, 1].ravel()
    conn = quad_connectivity(nM, Nm)
    ncell = conn.shape[0]
    cells = np.empty((ncell, 5), dtype=">i4")
    cells[:, 0] = 4
    cells[:, 1:] = conn
    with open(path, "wb") as f:
        f.write(b"# vtk DataFile Version 3.0\n")
        f.write(title.encode()[:255] + b"\n")
        f.write(b"BINARY\nDATASET UNSTRUCTURED_GRID\n")
        f.write(f"POINTS {npts} float\n".encode())
        f.write(pts.tobytes())
        f.write(f"\nCELLS {ncell} {ncell * 5}\n".encode())
        f.write(cells.tobytes())
        f.write(f"\nCELL_TYPES {ncell}\n".encode())
        f.write(np.full(ncell, VTK_QUAD, dtype=">i4").tobytes())
        f.write(f"\nPOINT_DATA {npts}\nSCALARS v float 1\nLOOKUP_TABLE default\n".encode())
        f.write(xyv[:, :, 2].ravel().astype(">f4").tobytes())
        f.write(b"\n")
