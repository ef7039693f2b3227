"""Register Sample Sort restated step by step (test infrastructure only).

Pure Python for small inputs.  Follows Sec. 3 of Bingmann, Marianczuk,
Sanders, "Engineering Faster Sorters for Small Sets of Items":

1. choose a sample of ``a*k`` items (oversampling factor ``a``) and sort it;
2. take the ``k-1`` splitters ``S_a, S_2a, ..., S_(k-1)a`` equidistant from the
   sorted sample, with the sentinels ``s_0 = -inf`` and ``s_k = +inf``;
3. classify every item into the bucket ``b_j`` with ``s_(j-1) < e <= s_j``,
   walking the splitters as a perfect binary tree stored in heap order
   ``t = [s_(k/2), s_(k/4), s_(3k/4), ...]``: from ``j = 1`` repeat
   ``j <- 2j + [t_j < e]`` log2(k) times (the "index built bit by bit" of
   Sec. 3.1);
4. finish every bucket of at most ``base`` items with the base-case sorter and
   recurse on larger ones.

Readings where the paper is silent (listed in the design notes):
* the sample is taken at the equidistant positions ``floor((2i+1)*len/(2*a*k))``;
* items are (key, original position) pairs compared lexicographically, so all
  items are distinct and equal keys cannot make a bucket repeat forever.
"""
from __future__ import annotations


def sample_positions(length: int, count: int) -> list[int]:
    """Equidistant sample positions (this library's reading; the paper leaves the choice open)."""
    return [((2 * i + 1) * length) // (2 * count) for i in range(count)]


def splitters_from_sample(sorted_sample: list, k: int, a: int) -> list:
    """s_1..s_(k-1) = S_a, S_2a, ..., S_(k-1)a with 1-based S (Sec. 3)."""
    return [sorted_sample[j * a - 1] for j in range(1, k)]


def heap_tree(splitters: list) -> list:
    """Heap-ordered perfect BST t[1..k-1] over s_1..s_(k-1) (Sec. 3.1); t[0] unused."""
    k = len(splitters) + 1
    t = [None] * k

    def fill(node: int, lo: int, hi: int) -> None:  # splitter indices lo..hi (1-based)
        if lo > hi:
            return
        mid = (lo + hi) // 2
        t[node] = splitters[mid - 1]
        fill(2 * node, lo, mid - 1)
        fill(2 * node + 1, mid + 1, hi)

    fill(1, 1, k - 1)
    return t


def classify_tree(e, tree: list) -> int:
    """0-based bucket index by the branch-free descent j <- 2j + [t_j < e]."""
    k = len(tree)
    j = 1
    while j < k:
        j = 2 * j + (1 if tree[j] < e else 0)
    return j - k


def classify_definition(e, splitters: list) -> int:
    """0-based bucket index straight from the definition s_(j-1) < e <= s_j."""
    k = len(splitters) + 1
    for j in range(1, k + 1):
        lower_ok = j == 1 or splitters[j - 2] < e
        upper_ok = j == k or e <= splitters[j - 1]
        if lower_ok and upper_ok:
            return j - 1
    raise AssertionError("splitters not sorted")


def rss_sort(items: list, k: int = 4, a: int = 3, base: int = 16, base_sort=sorted) -> list:
    """Sort distinct, comparable items by Register Sample Sort with k buckets."""
    n = len(items)
    if n <= base:
        return list(base_sort(items))
    sample = [items[p] for p in sample_positions(n, a * k)]
    sample = list(base_sort(sample))
    spl = splitters_from_sample(sample, k, a)
    tree = heap_tree(spl)
    buckets = [[] for _ in range(k)]
    for e in items:
        buckets[classify_tree(e, tree)].append(e)
    out = []
    for b in buckets:
        if len(b) == n:  # cannot happen for distinct items and a*k <= n
            raise AssertionError("no progress")
        out.extend(rss_sort(b, k, a, base, base_sort))
    return out
