"""The seeded synthetic workloads follow the stated recipe (sizes, ranks, distributions,
seeds).  CPU only; the module holds inputs, no method arithmetic."""
import numpy as np

import workloads as wl


def test_workload_sizes_and_ranks():
    cases = {wl.tiny_nb2_l12(): (576, 1, 0), wl.mos2size_nb4_l36(): (20736, 1, 1024),
             wl.sweep_nb2_l24(): (2304, 256, 256), wl.prec_nb4_l48(): (36864, 64, 2048),
             wl.adj_nb2_l36(): (5184, 32, 512), wl.mos2size_channel(): (20736, 1, 65),
             wl.angle_nb4_l36(): (20736, 60, 1024)}
    for w, (N, B, r) in cases.items():
        assert (w.model.N, w.B, w.rank) == (N, B, r), w.name
        assert w.dt == 0.2
    # the mos2-size rank is ~5 % of N; the channel rank 5 % of Nk
    assert abs(wl.mos2size_nb4_l36().rank / 20736 - 0.05) < 0.002
    assert wl.mos2size_channel().rank == round(0.05 * 1296)


def test_seeded_pulse_distributions():
    pulses, steps = wl.draw_pulses(4096)
    E0 = np.array([p.E0 for p in pulses])
    om = np.array([p.omega for p in pulses])
    sg = np.array([p.sigma for p in pulses])
    st = np.array(steps)
    assert np.all((E0 >= 1e-4) & (E0 <= 1e-2)) and abs(np.log10(E0).mean() + 3.0) < 0.05
    assert np.all((om >= 0.06) & (om <= 0.16)) and np.all((sg >= 30.0) & (sg <= 120.0))
    assert st.min() >= 500 and st.max() <= 4000 and len(set(st.tolist())) > 1000
    assert all(p.t0 == 200.0 and p.kind == 0 for p in pulses)
    # same seed, same draw; the sweep's total work is fixed by the seed
    assert wl.draw_pulses(4096) == (pulses, steps)
    assert sum(wl.sweep_nb2_l24().steps) == 577218


def test_angle_sweep_directions_are_unit_vectors():
    w = wl.angle_nb4_l36()
    ang = [np.degrees(np.arctan2(p.dir_y, p.dir_x)) for p in w.pulses]
    assert np.allclose([p.dir_x ** 2 + p.dir_y ** 2 for p in w.pulses], 1.0)
    assert abs(ang[0] - 1.0) < 1e-9 and abs(ang[-1] - 60.0) < 1e-9
    assert all(p.kind == 2 and p.T_pulse == w.steps[0] * w.dt for p in w.pulses)


def test_early_pulses_recipe():
    """The early pulses of the batched comparisons: seeded, peaking within 60 steps of
    dt = 0.2, log-uniform amplitudes, unit field directions over a half turn."""
    a, b = wl.early_pulses(2048), wl.early_pulses(2048)
    assert a == b
    E0 = np.array([p.E0 for p in a])
    sg = np.array([p.sigma for p in a])
    ang = np.array([np.arctan2(p.dir_y, p.dir_x) for p in a])
    assert np.all((E0 >= 1e-4) & (E0 <= 1e-2)) and abs(np.log10(E0).mean() + 3.0) < 0.05
    assert np.all((sg >= 1.5) & (sg <= 3.0)) and all(p.t0 == 6.0 and p.kind == 0 for p in a)
    assert np.all((ang >= 0.0) & (ang <= np.pi)) and ang.max() - ang.min() > 3.0
    assert all(abs(p.dir_x ** 2 + p.dir_y ** 2 - 1.0) < 1e-12 for p in a)
    # the peak and two sigma of the envelope after it lie within 60 steps (12 time units)
    assert np.all(6.0 + 2.0 * sg <= 60 * 0.2)
