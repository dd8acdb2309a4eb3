// Host-side input: FASTA text to the ragged rows that motif_load_seqs_var takes.
//
// The paper searches uniform synthetic sequences of one length (Sec. IV.B) and names larger and
// real sequence data as future work (Sec. VI).  Real data comes as FASTA: records that start
// with a '>' header line, followed by sequence lines.  This parser keeps the residues of every
// record in order and leaves their interpretation (case, unknown symbols such as N) to the
// loader.
#include <stdint.h>
#include <string.h>

#include "motif_internal.h"

extern "C" int motif_fasta_parse(const char* text, int64_t text_len, char* seq_buf,
                                 int64_t buf_cap, int32_t* lengths, int32_t max_seqs,
                                 int32_t* n_out, int64_t* total_out) {
  if (!text || text_len < 0 || !n_out || !total_out || buf_cap < 0 || max_seqs < 0 ||
      (buf_cap > 0 && !seq_buf) || (max_seqs > 0 && !lengths))
    return MOTIF_ERR_ARG;
  int64_t n = 0, total = 0, cur = 0;  // records, residues, residues of the open record
  bool in_record = false;
  int64_t i = 0;
  while (i < text_len) {
    // One line: [i, e).
    int64_t e = i;
    while (e < text_len && text[e] != '\n') ++e;
    const char first = text[i];
    if (first == '>') {  // header: closes the open record and opens a new one
      if (in_record) {
        if (n <= max_seqs && n > 0) lengths[n - 1] = (int32_t)cur;
      }
      ++n;
      if (n > INT32_MAX) return MOTIF_ERR_ARG;
      in_record = true;
      cur = 0;
    } else if (first == ';') {
      // comment line of the original FASTA format
    } else {
      for (int64_t k = i; k < e; ++k) {
        const char c = text[k];
        if (c == ' ' || c == '\t' || c == '\r' || c == '\v' || c == '\f') continue;
        if (!in_record) return MOTIF_ERR_ARG;  // residues before the first header
        if (cur >= INT32_MAX) return MOTIF_ERR_ARG;
        if (total < buf_cap) seq_buf[total] = c;
        ++total;
        ++cur;
      }
    }
    i = e + 1;
  }
  if (in_record && n <= max_seqs) lengths[n - 1] = (int32_t)cur;
  *n_out = (int32_t)n;
  *total_out = total;
  return n > max_seqs || total > buf_cap ? MOTIF_ERR_CAPACITY : MOTIF_OK;
}
