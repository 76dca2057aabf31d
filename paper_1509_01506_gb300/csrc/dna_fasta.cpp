// dna_fasta.cpp -- FASTA ingest on the host: records, header lines and line breaks.
//
// A FASTA file holds records, each a '>' header line followed by sequence lines. The scan
// treats every non-base byte as a reset symbol, so a line break inside a record would
// break every match that spans it; the parser therefore joins each record's sequence
// lines into one contiguous run of bytes (bases and other letters kept as they are, case
// included) and reports where each record and each header begins and ends.

#include <cstdint>
#include <cstring>

#include "../../include/dna_dfa.h"

extern "C" int dna_fasta_parse(const char *text, uint64_t len, uint8_t *out, uint64_t cap, uint64_t *out_len,
                               uint64_t *rec_off, uint64_t *hdr_span, uint32_t rec_cap, uint32_t *n_records) {
    if ((!text && len) || !out_len || !n_records || (cap && !out)) return DNA_ERR_INVALID_ARG;
    uint64_t o = 0;
    uint32_t nr = 0;
    bool in_record = false;
    uint64_t i = 0;
    bool overflow = false;
    while (i < len) {
        if (text[i] == '>' && (i == 0 || text[i - 1] == '\n' || text[i - 1] == '\r')) {
            // a header line: the record's sequence starts after it
            uint64_t e = i + 1;
            while (e < len && text[e] != '\n' && text[e] != '\r') ++e;
            if (rec_off && nr < rec_cap) {
                rec_off[nr] = o;
                if (hdr_span) { hdr_span[2 * nr] = i + 1; hdr_span[2 * nr + 1] = e; }
            }
            ++nr;
            in_record = true;
            i = e;
            continue;
        }
        const char ch = text[i++];
        if (ch == '\n' || ch == '\r' || ch == ' ' || ch == '\t') continue;
        if (!in_record) {   // sequence text before any header: an unnamed first record
            if (rec_off && nr < rec_cap) {
                rec_off[nr] = o;
                if (hdr_span) { hdr_span[2 * nr] = 0; hdr_span[2 * nr + 1] = 0; }
            }
            ++nr;
            in_record = true;
        }
        if (out) {
            if (o < cap) out[o] = (uint8_t)ch;
            else overflow = true;
        }
        ++o;
    }
    if (rec_off && nr < rec_cap) rec_off[nr] = o;   // end of the last record
    *out_len = o;
    *n_records = nr;
    if (overflow || (rec_off && nr + 1 > rec_cap)) return DNA_ERR_CAPACITY;
    return DNA_OK;
}
