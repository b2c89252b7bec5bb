"""The sequential drivers' choice of the next round's proposal, restated
from the rounds they report (checked against what they did)."""


def flow_is_kept(r, ess_min, rule="efficiency"):
    """The fallback rules. By efficiency: a flow round keeps the flow when its
    effective samples per simulation reach the acceptance rate of its own
    defensive prior draws; a prior round switches to the flow when its ESS
    fraction reaches ess_min. By ESS: every round by its ESS fraction. Fewer
    than 64 accepted samples mean the prior."""
    if r["n_accepted"] < 64:
        return 0
    if rule == "ess" or r["proposal"] == 0 or r["n_defensive"] == 0:
        return int(r["ess_fraction"] >= ess_min)
    ess = r["ess_fraction"] * r["n_accepted"]
    return int(ess / r["n_sims"] >= r["n_defensive_accepted"] / r["n_defensive"])
