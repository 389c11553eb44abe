"""Helpers of the GPU parity tests: host-side views of device results (no method arithmetic)."""
import numpy as np

import paper_1412_3228_gb300 as hom


def dense_ctilde(mat, cell_index, fp64=True):
    """Packed c~ [n^dim, ns] of one cell, expanded on the host from labels and tables."""
    off = mat.voxel_offsets()[cell_index]
    c = mat.cells[cell_index]
    nv = c.n ** c.dim
    lab = mat.label[off:off + nv].cpu().numpy().view(np.uint32).astype(np.int64)
    ns = hom.ns_of(mat.dim)
    tp = (mat.phase_c64 if fp64 else mat.phase_c32).cpu().numpy().reshape(-1, ns)
    tm = (mat.mixed_c64 if fp64 else mat.mixed_c32).cpu().numpy().reshape(-1, ns)
    mixed = (lab & hom.HOM_MIXED_BIT) != 0
    idx = lab & 0x7FFFFFFF
    out = np.empty((nv, ns), dtype=tp.dtype)
    out[~mixed] = tp[idx[~mixed]]
    out[mixed] = tm[idx[mixed]]
    return out, mixed


def unpack(packed, nc):
    """[..., ns] packed upper triangle -> [..., nc, nc] symmetric."""
    out = np.zeros(packed.shape[:-1] + (nc, nc), dtype=packed.dtype)
    k = 0
    for i in range(nc):
        for j in range(i, nc):
            out[..., i, j] = packed[..., k]
            out[..., j, i] = packed[..., k]
            k += 1
    return out


def cell_fields(res, cells, dim, key):
    """Split a flat output field into per-cell numpy arrays [L, nc, (n,) n, n]."""
    nc = hom.nc_of(dim)
    f = res[key].cpu().numpy()
    out, off = [], 0
    for c in cells:
        size = res["L"] * nc * c.n ** c.dim
        out.append(f[off:off + size].reshape((res["L"], nc) + (c.n,) * c.dim))
        off += size
    return out
