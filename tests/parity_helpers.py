"""Helpers shared by the GPU parity tests (test infrastructure: imports the oracle)."""
from oracle import oracle as O

# rounding-level perturbations of the input: x -> a x + b, undone on the
# outputs by the exact homogeneity of 1/r (pot scales by 1/a, grad by 1/a^2)
INPUT_MAPS = ((3.0, 0.1234567), (0.7, -0.3141592))


def rounding_floor(x, q, p, M, pot_o, grad_o, **kw):
    """How far two correct FP64 evaluations of the method can lie apart,
    measured on the oracle itself as the worst of
      * its change when its operators are recomputed as another correct FP64
        implementation might (oracle.operators_perturbed: the backward error
        of the SVD, one-ulp translation entries; two seeds), and
      * its change when the input is rounded differently (x -> a x + b, which
        moves every coordinate by up to one unit in its last place, undone
        exactly on the outputs), the GPU path's own situation: it works on
        leaf-relative offsets in root-normalised units, a re-rounding of the
        caller's coordinates.
    The GPU path (another SVD, composite operators, other summation orders) is
    held to 10x this floor, and never looser than 1e-12 where it is smaller.
    `kw` may hold a frozen tree and its lists; the tree is mapped with the
    particles."""
    fp = fg = 0.0
    for seed in (1, 2):
        po, go, _ = O.kifmm(x, q, p=p, leaf_cap=M, ops=O.operators_perturbed(p, seed), **kw)
        fp = max(fp, O.rel_l2(po, pot_o))
        fg = max(fg, O.rel_l2(go, grad_o))
    for a, b in INPUT_MAPS:
        kw_m = dict(kw)
        if "tree" in kw:  # a frozen tree maps with its particles (root cube a lo + b, side a side)
            t = dict(kw["tree"])
            t["lo"] = a * t["lo"] + b
            t["side"] = a * t["side"]
            kw_m["tree"] = t
        po, go, _ = O.kifmm(a * x + b, q, p=p, leaf_cap=M, **kw_m)
        fp = max(fp, O.rel_l2(a * po, pot_o))
        fg = max(fg, O.rel_l2(a * a * go, grad_o))
    return max(1e-12, 10 * fp), max(1e-12, 10 * fg)


def periodic_rounding_floor(x, q, L, p, M, pot_o, grad_o):
    """The same for the periodic method (oracle.kifmm_periodic): its change
    under the operator perturbation (two seeds) and under a scaling of the
    whole cell, x -> a x and L -> a L (a translation would move particles
    across the cell boundary, which changes the tree, not just the rounding).
    The periodic potential reads the root's equivalent density through the
    far-image operator and the second-moment term, so it inherits the
    pseudo-inverse's conditioning: at p = 6 two correct FP64 evaluations
    differ by ~1e-8 in the potential and ~2e-10 in the gradient."""
    fp = fg = 0.0
    for seed in (1, 2):
        po, go = O.kifmm_periodic(x, q, L, p=p, leaf_cap=M, ops=O.operators_perturbed(p, seed))
        fp = max(fp, O.rel_l2(po, pot_o))
        fg = max(fg, O.rel_l2(go, grad_o))
    for a in (3.0, 0.7):
        po, go = O.kifmm_periodic(a * x, q, a * L, p=p, leaf_cap=M)
        fp = max(fp, O.rel_l2(a * po, pot_o))
        fg = max(fg, O.rel_l2(a * a * go, grad_o))
    return max(1e-12, 10 * fp), max(1e-12, 10 * fg)
