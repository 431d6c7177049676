"""Host logic of the batch autotuner (no GPU): the trial sample and the cache signature."""
from paper_0908_4520_gb300 import autotune, inputs


def _cls(d):
    return (d["quadrature"], d["n_eq"], d["nx"] * d["ny"])


def test_sample_holds_the_whole_mix():
    """A trial runs the whole mix (up to 1024 instances), so it fills every SM the way the
    real launch does."""
    inst = inputs.batch_instances(512)
    smp = autotune._sample(inst, 1024)
    assert len(smp) == len(inst)
    assert sorted(d["id"] for d in smp) == list(range(len(inst)))


def test_small_sample_takes_one_instance_per_class_first():
    inst = inputs.batch_instances(512)
    classes = []
    for d in inst:
        if _cls(d) not in classes:
            classes.append(_cls(d))
    k = 12
    smp = autotune._sample(inst, k)
    assert len(smp) == k
    assert [_cls(d) for d in smp] == classes[:k]


def test_signature_depends_on_the_classes_and_storage_only():
    inst = inputs.batch_instances(64)
    s = autotune._signature(inst, "f32")
    assert s.startswith("f32:")
    assert autotune._signature(list(reversed(inst)), "f32") == s
    assert autotune._signature(inst, "f16") != s
    assert autotune._signature(inst[:8], "f32") != s
    assert all(len(c) == 3 for c in autotune.CANDIDATES)
