"""The early-exit cull grid is conservative (host only, no GPU).

For random obstacle sets and link-ball radius R, every point whose float32
cell lookup (as the kernels compute it) lands in a cell must find there the
pair bit of every obstacle it can reach (sphere: distance < R + r, box:
distance < R, exact in float64); a point outside the grid must reach none.
Points just inside each obstacle's reach probe the boundaries."""
import numpy as np
import pytest

from paper_2608_25830_b300 import binding


def _obstacles(rng, n_s, n_b):
    sp = np.concatenate([rng.uniform(-0.75, 0.75, (n_s, 3)), rng.uniform(0.05, 0.15, (n_s, 1))], axis=1)
    c = rng.uniform(-0.75, 0.75, (n_b, 3))
    h = rng.uniform(0.05, 0.15, (n_b, 3))
    bx = np.concatenate([c - h, c + h], axis=1)
    return sp.astype(np.float32), bx.astype(np.float32)


def _lookup(P, masks, origin, inv):
    nz, ny, nx = masks.shape
    f = (P - origin[None, :]) * inv                      # float32, as the kernels round it
    dims = np.array([nx, ny, nz], np.float32)
    inside = np.all((f >= 0) & (f < dims[None, :]), axis=1)
    idx = np.minimum(np.floor(np.where(inside[:, None], f, 0)).astype(np.int64), np.array([nx, ny, nz]) - 1)
    out = np.zeros(P.shape[0], np.uint64)
    out[inside] = masks[idx[inside, 2], idx[inside, 1], idx[inside, 0]]
    return out


def _needed(P, sp, bx, R):
    P64 = P.astype(np.float64)
    n_sp = (sp.shape[0] + 1) // 2
    need = np.zeros(P.shape[0], np.uint64)
    for o in range(sp.shape[0]):
        d = np.linalg.norm(P64 - sp[o, :3].astype(np.float64), axis=1)
        need |= np.where(d < R + float(sp[o, 3]), np.uint64(1) << np.uint64(o // 2), np.uint64(0))
    for o in range(bx.shape[0]):
        lo, hi = bx[o, :3].astype(np.float64), bx[o, 3:].astype(np.float64)
        gap = np.maximum(np.maximum(lo - P64, P64 - hi), 0.0)
        d = np.linalg.norm(gap, axis=1)
        need |= np.where(d < R, np.uint64(1) << np.uint64(n_sp + o // 2), np.uint64(0))
    return need


@pytest.mark.parametrize("n_s,n_b,seed", [(20, 10, 0), (26, 14, 1), (5, 0, 2), (0, 7, 3), (40, 24, 4)])
def test_cull_grid_is_conservative(n_s, n_b, seed):
    rng = np.random.default_rng(seed)
    sp, bx = _obstacles(rng, n_s, n_b)
    R = np.float32(0.2)
    masks, origin, inv = binding.gtmp_cull_grid(sp, bx, R)
    assert masks.size > 0
    P = [rng.uniform(-1.6, 1.6, (20000, 3))]
    for o in range(n_s):                                   # just inside each sphere's reach
        u = rng.normal(size=(200, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        P.append(sp[o, :3] + u * (float(R) + float(sp[o, 3]) - 1e-5))
    for o in range(n_b):                                   # just inside each box's reach, off a face
        u = rng.normal(size=(200, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        c = 0.5 * (bx[o, :3] + bx[o, 3:])
        h = 0.5 * (bx[o, 3:] - bx[o, :3])
        P.append(c + np.clip(u * 10.0, -h, h) + u * (float(R) - 1e-5))
    P = np.concatenate(P).astype(np.float32)
    got = _lookup(P, masks, origin, inv)
    need = _needed(P, sp, bx, float(R))
    missing = need & ~got
    assert not missing.any(), np.nonzero(missing)[0][:5]
    # and it prunes: most cells keep few pairs
    pairs = (n_s + 1) // 2 + (n_b + 1) // 2
    pop = np.unpackbits(masks.view(np.uint8)).reshape(masks.size, 32).sum(axis=1)
    assert pop.mean() < 0.25 * pairs


def test_cull_grid_absent_beyond_32_pairs_and_without_obstacles():
    rng = np.random.default_rng(9)
    sp, bx = _obstacles(rng, 40, 30)                       # 20 + 15 = 35 pairs
    masks, _, _ = binding.gtmp_cull_grid(sp, bx, 0.2)
    assert masks.size == 0
    masks, _, _ = binding.gtmp_cull_grid(np.zeros((0, 4)), np.zeros((0, 6)), 0.2)
    assert masks.size == 0
    with pytest.raises(binding.GtmpError):
        binding.gtmp_cull_grid(sp[:4], bx[:2], -1.0)
