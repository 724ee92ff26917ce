"""Test helpers: zero crossings of a brick field along voxel edges."""
import numpy as np


def dense_from_bricks(vals, bricks, n):
    """Scatter per-voxel values (brick order, x fastest in a brick) into an (n, n, n) [z, y, x] grid."""
    li = np.arange(512)
    loc = np.stack([li % 8, (li // 8) % 8, li // 64], axis=1)
    g = (8 * np.asarray(bricks)[:, None, :] + loc[None]).reshape(-1, 3)
    out = np.zeros((n, n, n), dtype=np.asarray(vals).dtype)
    out[g[:, 2], g[:, 1], g[:, 0]] = np.asarray(vals).reshape(-1)
    return out


def edge_crossings(U, mask, h, origin=(0.0, 0.0, 0.0), eps=0.0):
    """World positions of sign changes of U on voxel edges whose endpoints are both in `mask`.

    Linear interpolation along the edge; endpoints with |U| <= eps are skipped.
    Returns (positions (k, 3) xyz, edge ids (axis, z, y, x) (k, 4)).
    """
    pos, ids = [], []
    for ax in range(3):  # array axis: 0=z, 1=y, 2=x
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = slice(0, -1)
        sl1[ax] = slice(1, None)
        a, b = U[tuple(sl0)], U[tuple(sl1)]
        m = (np.sign(a) * np.sign(b) < 0) & mask[tuple(sl0)] & mask[tuple(sl1)] & (np.abs(a) > eps) & (np.abs(b) > eps)
        idx = np.nonzero(m)
        t = a[idx] / (a[idx] - b[idx])
        zyx = np.stack(idx, 1).astype(np.float64)
        zyx[:, ax] += t
        xyz = (zyx[:, ::-1] + 0.5) * h + np.asarray(origin)
        pos.append(xyz)
        ids.append(np.concatenate([np.full((len(t), 1), ax), np.stack(idx, 1)], 1))
    return np.concatenate(pos), np.concatenate(ids)
