"""Element-aggregate hierarchies by recursive coordinate bisection (RCB).

The paper forms its nested aggregates with METIS on the element face graph
(Section 4.1): the coarsest level has 2^d aggregates and every aggregate is
split into 2^d parts until single elements remain.  METIS is not available
here; this recipe stands in for it with a deterministic RCB order of the
element centroids:

* rcb_order(S): if |S| <= 1 return S; pick the axis of largest bounding-box
  extent over S (lowest axis on ties); stable-sort S by (centroid[axis],
  element id); the left half is the first ceil(|S|/2) elements; recurse.
* the level-k aggregate of element e is floor(pos(e) / (2^d)^k), so levels
  nest and each aggregate is 2^d aggregates of the level above.

Every split of a level is processed at once (vectorised), not recursively.
"""
import numpy as np


def rcb_order(centroids: np.ndarray) -> np.ndarray:
    n, d = centroids.shape
    order = np.arange(n)
    seg_start = np.array([0])
    seg_len = np.array([n])
    while True:
        active = seg_len > 1
        if not np.any(active):
            break
        seg_id = np.repeat(np.arange(seg_start.size), seg_len)
        c = centroids[order]
        lo = np.minimum.reduceat(c, seg_start, axis=0)
        hi = np.maximum.reduceat(c, seg_start, axis=0)
        ext = hi - lo
        axis = np.argmax(ext, axis=1)               # first maximum = lowest axis on ties
        key = c[np.arange(n), axis[seg_id]]
        o = np.lexsort((order, key, seg_id))        # stable by (segment, value, id)
        order = order[o]
        left = (seg_len + 1) // 2
        right = seg_len - left
        ns = np.stack([seg_start, seg_start + left], axis=1).ravel()
        nl = np.stack([left, right], axis=1).ravel()
        keep = nl > 0
        seg_start, seg_len = ns[keep], nl[keep]
    return order


def chunk_hierarchy(order: np.ndarray, dim: int, n_levels: int):
    """agg_of[k-1][i] = level-k aggregate of level-(k-1) unit i, k = 1..N,
    where N = n_levels - 1 (levels L0 .. LN)."""
    n = order.size
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    fan = 2 ** dim
    aggs = []
    # level-k aggregate of element e is pos(e) // fan^k; level-0 units are elements
    lvl_prev_of_elem = np.arange(n)
    for k in range(1, n_levels):
        lvl_of_elem = pos // fan ** k
        n_prev = int(lvl_prev_of_elem.max()) + 1
        a = np.empty(n_prev, dtype=np.int64)
        a[lvl_prev_of_elem] = lvl_of_elem
        aggs.append(a.astype(np.int32))
        lvl_prev_of_elem = lvl_of_elem
    return aggs


def paper_level_count(n_elems: int, dim: int) -> int:
    """Levels L0..LN with N+1 = ceil(log_{2^d} |T_h|) (Section 6 opening)."""
    fan = 2 ** dim
    N1, m = 0, 1
    while m < n_elems:
        m *= fan
        N1 += 1
    return max(N1, 2)
