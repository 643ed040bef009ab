"""The seeded input generator (no method arithmetic): determinism, the
shapes of the study templates and the layout of the study tomograms."""
import numpy as np

from paper_2408_02398_gb300 import synth


def test_generator_is_deterministic_and_seeded():
    a = synth.normals(7, synth.STREAM_NOISE, 1000)
    b = synth.normals(7, synth.STREAM_NOISE, 1000)
    c = synth.normals(8, synth.STREAM_NOISE, 1000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(a.mean()) < 0.1 and abs(a.std() - 1) < 0.1
    q = synth.shoemake_quats(synth.uniforms(3, synth.STREAM_ROT, 300))
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0)


def test_cylinder_is_a_cylinder():
    t = synth.cylinder_template(21)
    assert t.shape == (21, 21, 21) and t.max() == 1.0
    # invariant under quarter turns about z and the flip z -> -z (about the centre)
    assert np.array_equal(t, np.rot90(t, 1, axes=(1, 2)))
    assert np.array_equal(t, t[::-1])
    # solid on the axis over its length, empty beyond it
    assert t[10, 10, 10] == 1.0 and t[10 + 6, 10, 10] == 1.0 and t[10 + 9, 10, 10] == 0.0
    assert t[10, 10, 10 + 5] == 0.0


def test_l_shape_is_centred_and_without_rotational_symmetry():
    t = synth.l_shape_template(21)
    g = np.arange(21) - 10
    m = t.sum()
    com = [float((t.sum(axis=(1, 2)) * g).sum() / m), float((t.sum(axis=(0, 2)) * g).sum() / m),
           float((t.sum(axis=(0, 1)) * g).sum() / m)]
    assert np.abs(com).max() < 0.1
    # no half or quarter turn about a grid axis maps it onto itself
    for axes in ((0, 1), (0, 2), (1, 2)):
        for k in (1, 2, 3):
            assert not np.allclose(t, np.rot90(t, k, axes=axes), atol=1e-3)


def test_grid_tomogram_layout_and_snr():
    t = synth.l_shape_template(21).astype(np.float32)
    vol, pl = synth.grid_tomogram(t, 5, 26, 6, 31, None, 9.0)
    assert vol.shape == (137, 137, 137) and len(pl.centres) == 125
    c = np.asarray(pl.centres)
    assert c.min() == 6 + 10 and c.max() == 6 + 10 + 4 * 26
    # noise-free: each copy's window holds the template's mass, the gaps are empty
    z, y, x = (int(v) for v in c[0])
    assert abs(vol[z - 10:z + 11, y - 10:y + 11, x - 10:x + 11].sum() - t.sum()) < 0.05 * t.sum()
    assert vol[:5].max() == 0.0
    noisy, _ = synth.grid_tomogram(t, 5, 26, 6, 31, 0.5, 9.0)
    m = synth.sphere_mask_values(21, 9.0)
    sig2 = float(np.var(t.astype(np.float64)[m])) / 0.5
    assert abs(np.var(noisy[:5]) - sig2) < 0.05 * sig2
