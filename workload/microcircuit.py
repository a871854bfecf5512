"""The Potjans-Diesmann microcircuit as the paper states it (§2.2), as plain data.

Every number below is typed from the paper's tables:

* Table "params" (general and simulation parameters, §2.2): dt, C_m, tau_m, tau_ref,
  tau_syn, u_rest (= u_reset), u_thr, nu_th, omega_ext.
* Table "params2" (population-specific parameters, §2.2): N_i, thalamic in-degree K_i,
  initial-potential Gaussians, synaptic-amplitude Gaussians and delay Gaussians, plus
  the caption's doubled pathway.
* Table "params3" (connection probabilities, §2.2).

Readings where the paper is ambiguous:

* Connection table orientation: rows are the *target* population and columns the
  *source* population (the PD model the paper reproduces via NEST, §4.1). The caption's
  "rows = source" wording is not followed. ``Model.conn_p[target][source]``.
* The doubled pathway "L23/exh to L3/exh" (caption of Table params2) is L4E -> L23E,
  amplitude N(0.3, 0.03) mV.
* The inhibitory delay Gaussian is N(0.75, 0.375) ms (relative SD 0.5 as for the
  excitatory one) instead of the printed 0.325.
* All N(mu, s) entries are (mean, standard deviation).
* Amplitudes and delays are properties of the *source* population (its row in
  Table params2).

No arithmetic of the method is here: this module only carries numbers.
"""

from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

POP_NAMES = ("L23E", "L23I", "L4E", "L4I", "L5E", "L5I", "L6E", "L6I")

# Table params2, column N_i (full-scale population sizes).
_N_FULL = (20683, 5834, 21915, 5479, 4850, 1065, 14395, 2948)
# Table params2, column K (thalamic in-degree per neuron).
_K_EXT = (1600, 1500, 2100, 1900, 2000, 1900, 2900, 2100)
# Table params2, column u_init: N(mean, sd) in mV.
_U0 = ((-68.28, 5.36), (-63.16, 4.57), (-63.33, 4.74), (-63.45, 4.94),
       (-63.11, 4.94), (-61.66, 4.55), (-66.72, 5.46), (-61.43, 4.48))
# Table params2, column omega_i: synaptic amplitude N(mean, sd) in mV, by source pop.
_W_EXC = (0.15, 0.015)
_W_INH = (-0.6, 0.06)
# Table params2, column delta_i: delay N(mean, sd) in ms, by source pop.  The
# inhibitory SD follows the reading above (0.375, not the printed 0.325).
_D_EXC = (1.5, 0.75)
_D_INH = (0.75, 0.375)
_D_INH_PRINTED_SD = 0.325

# Table params3 exactly as printed: printed_row r, printed_column c, both in POP_NAMES order.
_CONN_PRINTED = (
    (0.1009, 0.1689, 0.0437, 0.0818, 0.0323, 0.0000, 0.0076, 0.0000),
    (0.1346, 0.1371, 0.0316, 0.0515, 0.0755, 0.0000, 0.0042, 0.0000),
    (0.0077, 0.0059, 0.0497, 0.1350, 0.0067, 0.0003, 0.0453, 0.0000),
    (0.0691, 0.0029, 0.0794, 0.1597, 0.0033, 0.0000, 0.1057, 0.0000),
    (0.1004, 0.0622, 0.0505, 0.0057, 0.0831, 0.3726, 0.0204, 0.0000),
    (0.0548, 0.0269, 0.0257, 0.0022, 0.0600, 0.3158, 0.0086, 0.0000),
    (0.0156, 0.0066, 0.0211, 0.0166, 0.0572, 0.0197, 0.0396, 0.2252),
    (0.0364, 0.0010, 0.0034, 0.0005, 0.0277, 0.0080, 0.0658, 0.1443),
)


@dataclass
class Model:
    """Parameters of one circuit.  Units: ms, pF, mV, Hz."""

    n_pops: int = 8
    # Table params
    dt_ms: float = 0.1
    C_m_pF: float = 250.0
    tau_m_ms: float = 10.0
    tau_ref_ms: float = 2.0
    tau_syn_ms: float = 0.5
    u_rest_mV: float = -65.0
    u_reset_mV: float = -65.0
    u_thr_mV: float = -50.0
    nu_th_hz: float = 8.0
    w_ext_mV: float = 0.15
    # Table params2 (per population, POP_NAMES order)
    n_full: List[int] = field(default_factory=lambda: list(_N_FULL))
    k_ext: List[float] = field(default_factory=lambda: [float(k) for k in _K_EXT])
    u0_mean_mV: List[float] = field(default_factory=lambda: [m for m, _ in _U0])
    u0_sd_mV: List[float] = field(default_factory=lambda: [s for _, s in _U0])
    w_mean_mV: List[float] = field(
        default_factory=lambda: [(_W_EXC if i % 2 == 0 else _W_INH)[0] for i in range(8)])
    w_sd_mV: List[float] = field(
        default_factory=lambda: [(_W_EXC if i % 2 == 0 else _W_INH)[1] for i in range(8)])
    d_mean_ms: List[float] = field(
        default_factory=lambda: [(_D_EXC if i % 2 == 0 else _D_INH)[0] for i in range(8)])
    d_sd_ms: List[float] = field(
        default_factory=lambda: [(_D_EXC if i % 2 == 0 else _D_INH)[1] for i in range(8)])
    # Table params3, read as conn_p[target][source]
    conn_p: List[List[float]] = field(
        default_factory=lambda: [list(row) for row in _CONN_PRINTED])
    # (source, target, mean mV, sd mV) amplitude overrides: the doubled pathway L4E -> L23E
    overrides: List[Tuple[int, int, float, float]] = field(
        default_factory=lambda: [(2, 0, 0.3, 0.03)])

    def replace(self, **kw) -> "Model":
        return dataclasses.replace(self, **kw)


def microcircuit_model(conn_orientation: str = "row_is_target",
                       inh_delay_sd_ms: float = _D_INH[1]) -> Model:
    """The paper's microcircuit.  ``conn_orientation='row_is_source'`` transposes
    Table params3 (the caption's literal wording); ``inh_delay_sd_ms=0.325`` gives the
    printed inhibitory delay SD."""
    m = Model()
    if conn_orientation == "row_is_source":
        m.conn_p = [[_CONN_PRINTED[s][t] for s in range(8)] for t in range(8)]
    elif conn_orientation != "row_is_target":
        raise ValueError(conn_orientation)
    m.d_sd_ms = [(_D_EXC[1] if i % 2 == 0 else inh_delay_sd_ms) for i in range(8)]
    return m


@dataclass(frozen=True)
class Workload:
    """A named run: circuit scale (integer permille of neurons and of in-degrees),
    network seed and number of 0.1 ms steps."""

    name: str
    scale_n_permille: int
    scale_k_permille: int
    seed: int
    steps: int
    description: str = ""


WORKLOADS = {
    # Tiny Potjans-Diesmann: 0.1x neurons, 0.1x in-degrees, 1,000 steps.
    "pd_tiny": Workload("pd_tiny", 100, 100, 1, 1000,
                        "PD microcircuit at 0.1x neurons (7,718) and 0.1x in-degrees (~2.85e6 synapses)"),
    # Full-scale microcircuit: 77,169 neurons, ~2.85e8 synapses, 10 s of biological time.
    "pd_full": Workload("pd_full", 1000, 1000, 1, 100000,
                        "PD microcircuit at full scale: 77,169 neurons, 284,811,022 synapses, 10 s"),
    # Scaled-up microcircuit: 4x neurons per population at full in-degrees, 1 s.
    "pd_x4": Workload("pd_x4", 4000, 1000, 1, 10000,
                      "PD microcircuit at 4x neurons (308,676) and full in-degrees (~1.14e9 synapses), 1 s"),
}


def batched_workloads(n_circuits: int = 32, master_seed: int = 2026,
                      steps: int = 20000) -> Sequence[Workload]:
    """Uneven circuits for the batched form: neuron and in-degree scales drawn uniformly
    from 100..1000 permille with numpy's Philox seeded by ``master_seed``; circuit c has
    network seed 1000 + c."""
    import numpy as np

    rng = np.random.Generator(np.random.Philox(master_seed))
    out = []
    for c in range(n_circuits):
        sn, sk = (int(x) for x in rng.integers(100, 1001, size=2))
        out.append(Workload(f"pd_batch_{c}", sn, sk, 1000 + c, steps))
    return out
