"""Oracle runs that the GPU tests hand to spawned worker processes, so that
the FP64 oracle advances its copy of a workload while the GPU runs the same
one (test infrastructure only; nothing here touches CUDA)."""


def full_run_diagnostics(cfg: dict, steps: int) -> dict:
    """Diagnostics (no spectrum) of the oracle after `steps` full steps."""
    import oracle
    s = oracle.Sim(cfg)
    s.step(steps)
    d = s.diagnostics()
    d.pop("spectrum", None)
    d["n_particles"] = s.np
    return d
