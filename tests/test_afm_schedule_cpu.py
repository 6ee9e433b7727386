"""run_host's choice between the overlapped and the one-stage forward (host logic only): the first
overlapped call is not timed, then the two schedules alternate until each has three timed calls,
and the one with the lower median is kept for good."""
import types

from paper_2401_14564_gb300 import afm


def fresh(overlap_ff=True):
    return types.SimpleNamespace(overlap_ff=overlap_ff, _mode=None, _trial={"overlap": [], "plain": []},
                                 _trial_warm=False, _TRIALS=afm.Simulator._TRIALS)


def drive(ns, times):
    seen = []
    for _ in range(12):
        mode = afm.Simulator._forward_mode(ns)
        seen.append(mode)
        afm.Simulator._note_forward(ns, mode == "overlap", times[mode])
    return seen


def test_faster_overlap_is_kept():
    ns = fresh()
    seen = drive(ns, {"overlap": 0.99, "plain": 1.16})
    assert seen[:8] == ["overlap", "overlap", "plain", "overlap", "plain", "overlap", "plain", "overlap"]
    assert ns._mode == "overlap" and set(seen[8:]) == {"overlap"}
    assert len(ns._trial["overlap"]) == 3 and len(ns._trial["plain"]) == 3


def test_faster_one_stage_forward_is_kept():
    ns = fresh()
    seen = drive(ns, {"overlap": 107.5, "plain": 103.9})
    assert ns._mode == "plain" and set(seen[7:]) == {"plain"}


def test_no_overlap_when_switched_off():
    ns = fresh(overlap_ff=False)
    assert set(drive(ns, {"overlap": 0.5, "plain": 1.0})) == {"plain"}
    assert ns._mode is None and ns._trial == {"overlap": [], "plain": []}
