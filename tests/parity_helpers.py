"""Helpers shared by the GPU parity tests (test infrastructure: imports the oracle)."""
from oracle import oracle as O


def rounding_floor(x, q, p, M, pot_o, grad_o, **kw):
    """The oracle's own change when its operators are recomputed as another
    correct FP64 implementation might (oracle.operators_perturbed: SVD
    backward error, one-ulp translation entries), worst of two seeds.  Two
    correct FP64 evaluations of the method lie this far apart; the GPU path
    builds its operators by another SVD (Jacobi) and applies them in
    composite form, so it is held to 10x this floor (and never looser than
    1e-12 where the floor is smaller)."""
    fp = fg = 0.0
    for seed in (1, 2):
        po, go, _ = O.kifmm(x, q, p=p, leaf_cap=M, ops=O.operators_perturbed(p, seed), **kw)
        fp = max(fp, O.rel_l2(po, pot_o))
        fg = max(fg, O.rel_l2(go, grad_o))
    return max(1e-12, 10 * fp), max(1e-12, 10 * fg)
