"""The ncu CSV summariser (paper_2406_06488_gb300/ncu_summary.py) on a small fixture in
ncu's `--csv --log-file` format: launch lists aggregate per kernel, metric captures
average per launch and turn the DRAM counters into traffic and a fraction of the
measured copy bandwidth."""
import pytest

from paper_2406_06488_gb300 import ncu_summary as ns

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
          '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"')


def _row(lid, kernel, metric, unit, value):
    return ('"%d","7","python3.12","127.0.0.1","%s","1","13","(576, 1, 1)","(152, 1, 1)","0","10.3",'
            '"Command line profiler metrics","%s","%s","%s"' % (lid, kernel, metric, unit, value))


LAUNCHES = "\n".join([
    "==PROF== Connected to process 7 (/usr/bin/python3.12)",
    HEADER,
    _row(0, "ept::k_masks(ept::Batch)", "gpu__time_duration.sum", "ns", "100000"),
    _row(1, "ept::<unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, ept::Batch)", "gpu__time_duration.sum",
         "ns", "300000"),
    _row(2, "void ept::k_pack<1>(ept::Batch)", "gpu__time_duration.sum", "usecond", "25"),
    _row(3, "ept::<unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, ept::Batch)", "gpu__time_duration.sum",
         "ns", "320,000"),
    _row(4, "ept::k_masks(ept::Batch)", "gpu__time_duration.sum", "ns", "140000"),
    "==PROF== Disconnected from process 7",
])

METRICS = "\n".join([
    HEADER,
    _row(0, "unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, Batch)", "dram__bytes_read.sum", "Mbyte", "59.0"),
    _row(0, "unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, Batch)", "dram__bytes_write.sum", "byte",
         "2000000"),
    _row(0, "unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, Batch)", "gpu__time_duration.sum", "usecond",
         "305"),
    _row(1, "unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, Batch)", "dram__bytes_read.sum", "Mbyte", "61.0"),
    _row(1, "unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, Batch)", "dram__bytes_write.sum", "byte",
         "2000000"),
    _row(1, "unnamed>::k_contract_tc(CUtensorMap_st, CUtensorMap_st, Batch)", "gpu__time_duration.sum", "usecond",
         "305"),
])


def test_kernel_names():
    assert ns.kernel_name("ept::k_masks(ept::Batch)") == "ept::k_masks"
    assert ns.kernel_name("void ept::k_pack<1>(ept::Batch)") == "ept::k_pack<1>"
    assert ns.kernel_name("unnamed>::k_contract_tc(CUtensorMap_st, Batch)") == "unnamed>::k_contract_tc"
    assert (ns.kernel_name("void at::vectorized_elementwise_kernel<4, at::FillFunctor<float>, std::array<char *, 1>>"
                           "(int, at::FillFunctor<float>, std::array<char *, 1>)")
            == "at::vectorized_elementwise_kernel<4, at::FillFunctor<float>, std::array<char *, 1>>")


def test_launch_list_aggregates_per_kernel():
    table = ns.launch_table(ns.read_rows(LAUNCHES))
    assert [t[0] for t in table] == ["ept::<unnamed>::k_contract_tc", "ept::k_masks", "ept::k_pack<1>"]
    contract, masks, pack = table
    assert contract[1] == 2 and contract[2] == pytest.approx(620.0) and contract[3] == pytest.approx(310.0)
    assert masks[1] == 2 and masks[2] == pytest.approx(240.0)
    assert pack[1] == 1 and pack[2] == pytest.approx(25.0)          # microseconds converted
    assert sum(t[4] for t in table) == pytest.approx(1.0)
    assert contract[4] == pytest.approx(620.0 / 885.0)
    md = ns.launches_markdown(table)
    assert md.splitlines()[2].startswith("| ept::<unnamed>::k_contract_tc | 2 | 620.0 | 310.0 | 70.1% |")


def test_metrics_traffic_and_bandwidth_fraction():
    table = ns.metric_table(ns.read_rows(METRICS), hbm_gbs=6766.0)
    d = table["unnamed>::k_contract_tc"]
    assert d["launches"] == 2
    assert d["dram__bytes_read.sum"] == pytest.approx(60.0)           # mean of the reported values
    assert d["traffic_bytes"] == pytest.approx(62.0e6)                 # units converted, per launch
    assert d["dram_gbs"] == pytest.approx(62.0e6 / 305e3)              # bytes per ns
    assert d["dram_frac"] == pytest.approx(62.0e6 / 305e3 / 6766.0)
    assert "| traffic_bytes | 6.2e+07 |" in ns.metrics_markdown(table)


def test_summarise_modes():
    assert "| ept::k_masks | 2 | 240.0 | 120.0 |" in ns.summarise("launches", LAUNCHES)
    assert "dram_frac" not in ns.summarise("metrics", METRICS)          # no peaks given
    assert "dram_frac" in ns.summarise("metrics", METRICS, hbm_gbs=6766.0)
    with pytest.raises(ValueError):
        ns.summarise("sections", LAUNCHES)


def test_phases_group_the_tuned_step():
    # per-launch means: contraction 310, draws 120, packing 25 (of 455 us)
    table = ns.phase_table(ns.read_rows(LAUNCHES))
    assert [(ph, ks) for ph, ks, _, _ in table] == [("contraction", ["k_contract_tc"]),
                                                    ("relabeling draws (side stream)", ["k_masks"]),
                                                    ("centring / packing", ["k_pack<1>"])]
    assert [round(us, 6) for _, _, us, _ in table] == [310.0, 120.0, 25.0]
    assert table[0][3] == pytest.approx(310.0 / 455.0)
    md = ns.summarise("phases", LAUNCHES)
    assert "| contraction | k_contract_tc | 310.0 | 68.1 % |" in md and md.splitlines()[-1] == "| total | | 455.0 | |"
