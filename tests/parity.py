"""Shared parity assertions of the GPU tests against the oracle."""


def assert_same_decisions(r, ref):
    """The second Gram-Schmidt pass (Fig. 1 steps 7-11) and the breakdown exit (step 12) taken as
    the oracle takes them: the same number of breakdowns, and second-pass counts that differ by no
    more than the Arnoldi step counts do (equal when the step counts are equal). A solve whose
    iteration count is within the 2% bar of the oracle's may take a few more or fewer steps, and
    on these systems almost every step takes the second pass, so its count moves with them; a
    decision taken differently on a step both runs share would show as a second-pass difference
    beyond the step difference."""
    assert r.breakdowns == ref.breakdowns, ("breakdowns", r.breakdowns, ref.breakdowns)
    assert abs(r.reorths - ref.reorths) <= abs(r.iters - ref.iters), \
        ("second passes", r.reorths, ref.reorths, "steps", r.iters, ref.iters)
