"""Every input recipe is a function of its seed: the same seed gives the same
images, flow and ground truth, another seed gives another scene; the batch
recipe keeps to its stated sizes and disparity counts; the confidence-training
renderer returns one pair per plane-recipe seed and two per automotive one."""
import numpy as np

from paper_1801_04720_gb300 import synth, train_confnet


def _same(a, b):
    return (all(np.array_equal(x, y) for x, y in zip(a.images(), b.images()))
            and np.array_equal(a.flow, b.flow) and np.array_equal(a.gt_disp0, b.gt_disp0))


def test_recipes_are_functions_of_the_seed():
    for make in (lambda s: synth.fronto_planes(seed=s),
                 lambda s: synth.automotive(seed=s, W=200, H=96, D=64, n_segments=4, disp_range=(2.0, 60.0)),
                 lambda s: synth.confidence_recipe(s, W=160, H=64, D=32)):
        assert _same(make(3), make(3))
        assert not _same(make(3), make(4))


def test_batch_recipe_sizes():
    sizes = {(320, 240), (640, 480), (1024, 320), (1242, 375)}
    for k in range(6):
        q = synth.batch_recipe(seed=k)
        H, W = q.shape
        assert (W, H) in sizes and q.D in (64, 128, 192)


def test_render_pairs_counts_and_shapes():
    planes = train_confnet.render_pairs([1, 2], 96, 40, 32, workers=2)
    auto = train_confnet.render_pairs([7], 96, 48, 32, recipe="automotive", workers=1)
    assert len(planes) == 2 and len(auto) == 2
    for left, right in planes + auto:
        assert left.dtype == np.uint8 and left.shape == right.shape
