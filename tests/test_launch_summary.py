"""Host-side tools of the measurement: parsing an ncu launch list, the
timed-region window, library names of device kernels, and the recorded
DRAM traffic being used only on the sources it was taken on."""
import json

from paper_2311_01598_gb300 import launch_summary as L

CSV = '''==PROF== Connected to process 123
"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","void at::native::elementwise_kernel<128, 2>(int, F)","1","7","(128, 1, 1)","(4, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","3.10"
"1","1","python","h","void ks::k_inv_row<ks::Shape<8, 8>>(ks::Tables, ks::LimbMaps)","1","7","(64, 1, 1)","(64, 384, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","120.5"
"2","1","python","h","void ks::(anonymous namespace)::k_bconv_tc<0, 1>(ks::Tables, ks::BUpJobs, ks::BDnJobs, const uint4 *, int, int, int, int)","1","7","(768, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ms","0.21"
"3","1","python","h","void ks::k_fwd_row<ks::Shape<8, 8>, false>(ks::Tables, ks::LimbMaps)","1","7","(64, 1, 1)","(64, 1152, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","300,000"
"4","1","python","h","void ks::k_fwd_row<ks::Shape<8, 8>, false>(ks::Tables, ks::LimbMaps)","1","7","(64, 1, 1)","(64, 768, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","ns","200,000"
"5","1","python","h","void ks::k_oc_comb_qw<false, 4>(ks::Tables, ks::OcJobs)","1","7","(256, 1, 1)","(64, 384, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","100"
'''


def test_read_launches_keeps_library_kernels_and_units(tmp_path):
    p = tmp_path / "launches.csv"
    p.write_text(CSV)
    rows = L.read_launches(str(p))
    assert [r[0] for r in rows] == ["k_inv_row<ks::Shape<8, 8>>", "k_bconv_tc<0, 1>", "k_fwd_row<ks::Shape<8, 8>, false>",
                                   "k_fwd_row<ks::Shape<8, 8>, false>", "k_oc_comb_qw<false, 4>"]
    assert [r[2] for r in rows] == [120500.0, 210000.0, 300000.0, 200000.0, 100000.0]


def test_summarise_window_and_shares(tmp_path):
    p = tmp_path / "launches.csv"
    p.write_text(CSV)
    rows = L.read_launches(str(p))
    table, total, n = L.summarise(rows, 1, 3)  # bconv, fwd_row, fwd_row
    assert n == 3 and total == 710000.0
    assert table[0][0] == "k_fwd_row<ks::Shape<8, 8>, false>" and table[0][1] == 2
    assert abs(sum(t[3] for t in table) - 1.0) < 1e-12
    md = L.to_markdown(table, total, n)
    assert "3 launches, 710.0 us total" in md and "| `k_bconv_tc<0, 1>` | 1 | 210.0 | 29.6% |" in md


def test_library_names():
    assert L.lib_name("void ks::(anonymous namespace)::k_bconv_tc<1, 1>(ks::Tables)") == "bconv_down"
    assert L.lib_name("void ks::(anonymous namespace)::k_bconv_tc<0, 2>(ks::Tables)") == "bconv_up"
    assert L.lib_name("void ks::(anonymous namespace)::k_bconv_tc<1, 1, 9>(ks::Tables)") == "bconv_down"
    assert L.lib_name("void ks::k_fwd_row<ks::Shape<8, 8>, true>(ks::Tables, ks::LimbMaps)") == "ntt_fwd_row"
    assert L.lib_name("void ks::k_oc_comb_qg<false, true, 2>(ks::Tables)") == "oc_comb_q"
    assert L.lib_name("void at::native::vectorized_elementwise_kernel<4>(int)") is None


def test_recorded_traffic_only_on_matching_sources(tmp_path, monkeypatch):
    rec = {"sources_sha256": L.kernel_sources_sha(), "capture": "ncu ...", "key_switches": 4,
           "kernels": {"ntt_fwd_row": {"launches": 2, "dram_bytes_per_ks": 127.0e6}}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(L, "TRAFFIC_PATH", str(p))
    assert L.recorded_traffic() == {"ntt_fwd_row": 127.0e6}
    rec["sources_sha256"] = "0" * 64
    p.write_text(json.dumps(rec))
    assert L.recorded_traffic() == {}
    monkeypatch.setattr(L, "TRAFFIC_PATH", str(tmp_path / "missing.json"))
    assert L.recorded_traffic() == {}
