"""The seeded input generators: fixed output for a fixed seed (the benchmarks
and parity tests of different runs and machines see the same series), the
documented construction, and the labelled shape-like classes."""

import hashlib

import numpy as np
import pytest

import synth


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:16]


def test_arithmetic_generators_are_pinned():
    # standard normals accumulated in fp64 and rounded once: platform-independent
    assert digest(synth.random_walks(50, 64, seed=1)) == "f1327df02976f6c8"
    assert digest(synth.white_noise(50, 64, seed=1)) == "551a874b7ef677a2"


def test_random_walk_construction():
    x = synth.random_walks(20, 100, seed=3).astype(np.float64)
    assert np.all(x[:, 0] == 0.0)
    steps = np.diff(x, axis=1).ravel()
    # N(0, 1) steps (rounding to fp32 aside)
    assert abs(steps.mean()) < 0.1 and abs(steps.std() - 1.0) < 0.1


def test_streams_and_seeds_differ():
    a = synth.random_walks(4, 32, seed=5)
    assert not np.array_equal(a, synth.random_walks(4, 32, seed=6))
    assert not np.array_equal(a, synth.random_walks(4, 32, seed=5, stream=synth.STREAM_QUERY))
    np.testing.assert_array_equal(a, synth.random_walks(4, 32, seed=5))


def test_shapes_are_z_normalised_and_repeatable():
    x = synth.shapes(40, 128, seed=2).astype(np.float64)
    np.testing.assert_allclose(x.mean(axis=1), 0.0, atol=1e-5)
    np.testing.assert_allclose(x.std(axis=1), 1.0, atol=1e-4)
    np.testing.assert_array_equal(synth.shapes(40, 128, seed=2), synth.shapes(40, 128, seed=2))


def test_shape_classes_follow_their_labels():
    labels = np.repeat(np.arange(synth.SHAPE_CLASSES), 25)
    x = synth.shape_classes(labels, 128, seed=4).astype(np.float64)
    assert x.shape == (100, 128) and x.dtype == np.float64
    np.testing.assert_allclose(x.mean(axis=1), 0.0, atol=1e-5)
    # plateaus and ramps have a long run of near-constant samples outside the
    # event; sums of sinusoids rarely do
    def flat_run(r):
        d = np.abs(np.diff(r)) < 0.5
        best = run = 0
        for v in d:
            run = run + 1 if v else 0
            best = max(best, run)
        return best

    runs = np.array([flat_run(r) for r in x])
    event = runs[labels < 3].mean()
    waves = runs[labels == 3].mean()
    assert event > waves, (event, waves)
    # rising ramps climb and falling ramps drop inside their event
    slope = np.array([np.polyfit(np.arange(128), r, 1)[0] for r in x])
    assert np.median(slope[labels == 1]) > np.median(slope[labels == 2])
    np.testing.assert_array_equal(synth.shape_classes(labels, 128, seed=4),
                                  synth.shape_classes(labels, 128, seed=4))


def test_shape_classes_reject_bad_labels():
    with pytest.raises(ValueError):
        synth.shape_classes([0, 4], 32, seed=1)
    with pytest.raises(ValueError):
        synth.shape_classes([[0, 1]], 32, seed=1)
