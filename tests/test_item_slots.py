"""The expansion's item order and the cell enumeration's link tables agree.

k_expand_vertices records the vertex-table slot of every coface item of an
edge (y, S) in item order: items r < 2^|S| - 2 are y + e(M) with M the
(r+1)-th subset of S (kind 0); after them, alternately, y + e(S) + e(M)
(kind 1) and y - e(M) (kind 2) for M the ((r - nsub) / 2 + 1)-th subset of
T = {0..d-1} minus S.  The cell enumeration's link table of the same edge
reads these slots: a[q] (q = compressed subset of S) is item q - 1, except
the edge's ends a[0] = y and a[2^|S| - 1] = y + e(S); b[r] and c[r] (r =
compressed subset of T) are items 2^|S| - 2 + 2 (r - 1) and the one after,
except b[0] = y + e(S) and c[0] = y.  This test restates both orders on the
host for every mask S at d = 2..7 and checks that each link-table entry maps
to the item with the same vertex."""


def _deposit(bits, mask):
    """The k-th set bit of mask takes bit k of bits (a compressed subset)."""
    out, k = 0, 0
    for i in range(32):
        if (mask >> i) & 1:
            if (bits >> k) & 1:
                out |= 1 << i
            k += 1
    return out


def _item(S, d, r):
    """(kind, M) of item r of edge mask S (the expansion's decode)."""
    nsub = (1 << bin(S).count("1")) - 2
    if r < nsub:
        return 0, _deposit(r + 1, S)
    r -= nsub
    T = ~S & ((1 << d) - 1)
    return 1 + (r & 1), _deposit((r >> 1) + 1, T)


def _vertex(S, kind, M):
    """The item's vertex as an offset from y: (+e(M)), (+e(S)+e(M)) or (-e(M))."""
    if kind == 0:
        return ("+", M)
    if kind == 1:
        return ("+", S | M)
    return ("-", M)


def test_link_table_entries_map_to_their_items():
    for d in range(2, 8):
        full = (1 << d) - 1
        for S in range(1, full + 1):
            T = ~S & full
            n1 = bin(S).count("1")
            na, nb = 1 << n1, 1 << (d - n1)
            count = (na - 2) + 2 * (nb - 1)
            items = [_vertex(S, *_item(S, d, r)) for r in range(count)]
            assert len(set(items)) == count  # distinct vertices
            for q in range(na):  # a[q] = y + e(deposit(q, S))
                want = ("+", _deposit(q, S))
                if q == 0 or q == na - 1:
                    continue  # the edge's ends: their signs come from the edge record
                assert items[q - 1] == want
            for r in range(1, nb):
                M = _deposit(r, T)
                assert items[(na - 2) + 2 * (r - 1)] == ("+", S | M)  # b[r]
                assert items[(na - 2) + 2 * (r - 1) + 1] == ("-", M)  # c[r]
