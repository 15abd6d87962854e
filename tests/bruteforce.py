"""Brute-force local-alignment score by enumerating every alignment (tiny inputs only).

Independent of any recurrence: an alignment is a start cell (i0, j0) plus a path of
operations M (consume one residue of each sequence, add SM), I (consume one subject
residue) and D (consume one query residue).  A gap run of k operations of one kind costs
goe + (k - 1) * ge; a run of I directly followed by a run of D (or the reverse) is two
runs, each opened.  The local score is the maximum over all start cells, all paths and
every prefix of every path, and over the empty alignment (0).  That is the textbook
definition of the best local alignment score with affine gaps.

Eqs. sw2-sw4 also let a run of one kind end and a new run of the same kind open right
after it (H includes E and F, and E/F re-open from H), so a continuing gap position may
be charged the opening cost instead of the extension cost.  That never helps when
goe >= ge; when goe < ge it does, so a continuing position costs min(ge, goe) here, as
it does in the equations.
"""


def local_score(q, d, sm, goe, ge):
    m, n = len(q), len(d)
    cont = min(ge, goe)
    best = 0

    def walk(i, j, score, last):
        nonlocal best
        if score > best:
            best = score
        if i < m and j < n:
            walk(i + 1, j + 1, score + int(sm[q[i]][d[j]]), "M")
        if j < n:
            walk(i, j + 1, score - (cont if last == "I" else goe), "I")
        if i < m:
            walk(i + 1, j, score - (cont if last == "D" else goe), "D")

    for i0 in range(m + 1):
        for j0 in range(n + 1):
            walk(i0, j0, 0, "")
    return best
