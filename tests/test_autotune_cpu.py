"""Host logic of the launch-shape autotuner (no GPU): the shape encoding and
the switching margin that keeps an incumbent shape against candidates whose
advantage is within the timing noise of short probes."""
from paper_2609_27342_gb300.autotune import pick, variant


def test_variant_encodes_one_choice_per_brick_kernel():
    seen = set()
    for p in range(3):
        for g in range(3):
            for f in range(3):
                v = variant(p, g, f)
                assert (v % 3, (v // 3) % 3, v // 9) == (p, g, f)
                seen.add(v)
    assert seen == set(range(27))


def test_pick_keeps_the_incumbent_within_the_margin():
    inc = {"relative": 1.0}
    near = {"relative": 0.995}
    far = {"relative": 0.98}
    slower = {"relative": 1.02}
    assert pick([inc, near], inc, 0.01) is inc
    assert pick([inc, near, far], inc, 0.01) is far
    assert pick([inc, slower], inc, 0.01) is inc
    assert pick([inc, near], None, 0.01) is near
    assert pick([inc, near], inc, 0.0) is near
