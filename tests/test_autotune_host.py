"""Host logic of the autotuner: its cache is keyed by everything that changes
which kernel builds a context runs (no GPU needed)."""
import copy
import types

import numpy as np


def test_variant_tags_and_signatures_differ():
    from paper_1909_05098_gb300.build import build
    build()
    from paper_1909_05098_gb300.autotune import signature, variant
    from synth.problem import Material, Perfusion
    from synth.scenarios import cube_hex_fp64
    base = cube_hex_fp64().problem
    info = {"elem_type": 8, "precision": 1, "n_nodes": base.n_nodes, "n_elems": len(base.conn), "n_free": 729,
            "n_convective": 0, "order": 0, "algorithmic_bytes_per_step": 123456}

    def solver(p, dose=False):
        return types.SimpleNamespace(problem=p, dose_model=dose)

    tab = copy.copy(base)
    tab.material = Material.tabulated((30.0, 70.0), (1060.0, 1000.0), (3600.0, 3300.0), (0.5, 0.7))
    reg = copy.copy(base)
    reg.regions, reg.region_materials, reg.region_perfusion = (np.zeros(len(base.conn), np.int32), (base.material,),
                                                               (Perfusion(),))
    full = copy.copy(base)
    full.hex_rule = "full"
    uni = copy.copy(base)
    uni.lumping = "uniform"
    sched = copy.copy(base)
    sched.schedule_end, sched.schedule_factor = np.array([1.0]), np.array([0.0])
    tags = [variant(solver(base)), variant(solver(tab)), variant(solver(reg)), variant(solver(full)),
            variant(solver(uni)), variant(solver(sched)), variant(solver(base, dose=True))]
    assert tags[0] == ""
    assert len(set(tags)) == len(tags), tags
    sigs = {signature(info, "GB300", t) for t in tags}
    assert len(sigs) == len(tags)
    assert signature(dict(info, algorithmic_bytes_per_step=1), "GB300") != signature(info, "GB300")
